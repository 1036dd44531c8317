// lee_api.cpp -- the C ABI of liblee (include/lee.h): context life cycle,
// arena layout, uploads, CUDA-graph stepping, read-back, checkpoints, batches.
// The library never allocates device memory: the caller passes one arena per
// context (and one per batch) sized by lee_plan / lee_batch_plan.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lee_internal.h"
#include "../../include/lee.h"

using namespace lee;

namespace {

thread_local std::string g_create_err;

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }
constexpr int GRAPH_STEPS = 8;

struct Layout {
    size_t q, mask, tiles, gt, gs, gn, gk, ei, ew, xn, xs, gx, gy, pi, pw, ph, clock, scratch, staging, desc,
        prefix, chunks, strips, tmap, bchunks, bc, ade, total;
};

// TMA stencil work list of one instance: columns of tiles (instance, tile
// column, first tile row, tiles), cut into segments of at most `seg` tiles so
// that small batches still give every SM work.  Inert tiles (all solid, no
// ghost: their outputs stay zero) at either end of a column are left out (the
// solid side of a straight wall: about half the tiles); inert tiles between
// live ones stay, so that a column is never split (on the cylinder sweep,
// splitting around the few tiles inside the cylinders cost 1.2 %).
void append_strips(std::vector<int4> &out, int inst, const InstDesc &d, int seg, const std::vector<uint32_t> &flags) {
    auto inert = [&](int tx, int ty) { return (flags[(size_t)ty * d.tiles_x + tx] & TILE_INERT) != 0; };
    for (int tx = 0; tx < d.tiles_x; ++tx) {
        int lo = 0, hi = d.tiles_y;
        while (lo < hi && inert(tx, lo)) ++lo;
        while (hi > lo && inert(tx, hi - 1)) --hi;
        for (int ty = lo; ty < hi; ty += seg) out.push_back(make_int4(inst, tx, ty, std::min(seg, hi - ty)));
    }
}
int strip_segment(long long total_tiles, int strips_per_sm = 2) {
    const long long n = (long long)strips_per_sm * num_sms();
    return (int)std::max<long long>(1, (total_tiles + n - 1) / n);
}
// longest strips first, dealt round-robin to the persistent CTAs
void sort_strips(std::vector<int4> &s) {
    std::stable_sort(s.begin(), s.end(), [](const int4 &a, const int4 &b) { return a.w > b.w; });
}

inline int n_chunks(int ng) { return (ng + GHOSTS_PER_CTA - 1) / GHOSTS_PER_CTA; }

// ghost work list of one instance: one entry per ghost CTA
void append_chunks(std::vector<int4> &out, int inst, int ng) {
    for (int c = 0; c < n_chunks(ng); ++c) {
        const int first = c * GHOSTS_PER_CTA;
        out.push_back(make_int4(inst, first, std::min(GHOSTS_PER_CTA, ng - first), 0));
    }
}

}  // namespace

namespace lee {
void set_global_error(const std::string &msg) { g_create_err = msg; }
}  // namespace lee

struct lee_ctx {
    lee_grid g{};
    Geometry geo;
    Impedance imp;
    double s_xs = 0, s_ys = 0, s_amp = 0, s_w = 1, s_omega = 0;
    std::vector<double> probe_xy;
    int probe_cap = 0;
    bool planned = false, bound = false;
    Plan plan;
    int kernel_mode = KERNEL_SMEM;
    Layout L{};
    char *dev = nullptr;
    cudaStream_t stream = nullptr;
    InstDesc hd{};
    InstDesc *dd = nullptr;
    int *dprefix = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // [0]: 1 step, [1]: GRAPH_STEPS steps
    long long graph_launches[2] = {0, 0};            // kernels per replay of each graph
    int nstrips = 0;
    int nband = 0;                    // band nodes redone by band_kernel (warp-specialised stencil)
    int nbchunks = 0;                 // their band_kernel work-list entries
    int tile_w_req = 0, tile_h_req = 0;   // lee_set_tile (0: the default shape)
    int sponge_w = 0;                 // lee_set_sponge: ramp width in cells (0: off)
    double sponge_k = 0.0;            // and strength kappa
    std::string err;
    size_t elem() const { return g.precision == LEE_FP32 ? 4 : 8; }
};

struct lee_batch {
    int precision = 0;
    std::vector<lee_ctx *> members;
    char *dev = nullptr;
    long long bytes = 0;
    cudaStream_t stream = nullptr;
    bool dirty = true;
    BatchView bv{};
    long long *status = nullptr;      // device: members' status words (lee_batch_status)
    int *probe_off = nullptr;         // device: offsets of the members' latest probe records
    double *probe_buf = nullptr;      // device: the latest probe records, side by side
    long long nprobe_values = 0;      // their total count
    int strips_per_sm = 2;            // lee_batch_set_strips_per_sm
    int fuse12 = 0;                   // lee_batch_set_stage_fusion
    int band_tile = -1;               // lee_batch_set_band_in_tile (-1: default_band_tile_stages())
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_launches[2] = {0, 0};
    std::string err;
};

namespace {

int fail(lee_ctx *c, int code, const std::string &m) { c->err = m; return code; }
int cuda_fail(lee_ctx *c, cudaError_t e, const char *what) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return LEE_ERR_CUDA;
}
#define CK(call)                                                   \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);   \
    } while (0)

void drop_graphs(cudaGraphExec_t g[2]) {
    for (int i = 0; i < 2; ++i)
        if (g[i]) { cudaGraphExecDestroy(g[i]); g[i] = nullptr; }
}

// band nodes redone by band_kernel (0 unless the stencil leaves the band to it)
int ctx_band_nodes(const lee_ctx *c) {
    const Plan &P = c->plan;
    return uses_band_pass(c->g.precision, c->kernel_mode, P.tile_w, P.tile_h)
               ? band_nodes(P.nx, P.ny, c->g.bc_x == LEE_BC_PERIODIC, c->g.bc_y == LEE_BC_PERIODIC)
               : 0;
}

Layout make_layout(const lee_ctx *c) {
    const Plan &P = c->plan;
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + std::max<size_t>(bytes, 1)); return at; };
    const size_t plane = (size_t)P.ny * P.pitch;
    const int ng = (int)P.g_target.size();
    const size_t ne = P.e_idx.size();
    const int np = (int)c->probe_xy.size() / 2;
    L.q = take(9 * plane * c->elem());
    L.mask = take(plane);
    L.tiles = take(P.tile_flags.size() * 4);
    L.gt = take((size_t)ng * 4);
    L.gs = take((size_t)(ng + 1) * 4);
    L.gn = take((size_t)ng * 16);
    L.gk = take((size_t)ng * 16);
    L.ei = take(ne * 4);
    L.ew = take(ne * 32);
    L.xn = take((size_t)ng * 8 * P.ns);
    L.xs = take((size_t)ng * 8 * P.ns);
    L.gx = take((size_t)P.nx * c->elem());
    L.gy = take((size_t)P.ny * c->elem());
    L.pi = take((size_t)np * 16 * 4);
    L.pw = take((size_t)np * 16 * 8);
    L.ph = take((size_t)np * std::max(c->probe_cap, 1) * 8);
    L.clock = take(8 * 8);
    L.scratch = take(64 * 8);
    L.staging = take((size_t)P.nx * P.ny * 8);
    L.desc = take(sizeof(InstDesc));
    L.prefix = take(8 * 4);
    L.chunks = take((size_t)(n_chunks(ng) + 1) * sizeof(int4));
    L.strips = take((size_t)(P.tiles_x * P.tiles_y + 1) * sizeof(int4));
    L.tmap = take(4 * 128);
    L.bchunks = take(((size_t)ctx_band_nodes(c) / 64 + 2) * sizeof(int4));
    L.bc = take((size_t)ng * 16);
    L.ade = take(P.ade_coef.size() * 8);
    L.total = o;
    return L;
}

void fill_source_profiles(const lee_ctx *c, std::vector<double> &gx, std::vector<double> &gy) {
    const Plan &P = c->plan;
    gx.assign(P.nx, 0.0);
    gy.assign(P.ny, 0.0);
    if (c->s_amp == 0.0) return;
    const double b = std::log(2.0) / (c->s_w * c->s_w);
    for (int i = 0; i < P.nx; ++i) { double d = c->g.x0 + i * c->g.h - c->s_xs; gx[i] = std::exp(-b * d * d); }
    for (int j = 0; j < P.ny; ++j) { double d = c->g.y0 + j * c->g.h - c->s_ys; gy[j] = std::exp(-b * d * d); }
}

int upload_source(lee_ctx *ctx) {
    std::vector<double> gx, gy;
    fill_source_profiles(ctx, gx, gy);
    if (ctx->g.precision == LEE_FP32) {
        std::vector<float> fx(gx.begin(), gx.end()), fy(gy.begin(), gy.end());
        CK(cudaMemcpyAsync(ctx->dev + ctx->L.gx, fx.data(), fx.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->dev + ctx->L.gy, fy.data(), fy.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        CK(cudaMemcpyAsync(ctx->dev + ctx->L.gx, gx.data(), gx.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->dev + ctx->L.gy, gy.data(), gy.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    }
    ctx->hd.s_amp = ctx->s_amp;
    ctx->hd.s_omega = ctx->s_omega;
    stage_forcing_factors(ctx->s_omega, ctx->hd.dt, ctx->hd.G_re, ctx->hd.G_im);
    CK(cudaMemcpyAsync(ctx->dd, &ctx->hd, sizeof(InstDesc), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

// Enqueue `steps` time steps of the instances in bv.
cudaError_t enqueue_steps(const BatchView &bv, int steps, cudaStream_t s) {
    static const int ctas = [] { const char *e = getenv("LEE_STENCIL_CTAS"); return e ? atoi(e) : 0; }();
    BatchView nb = bv;                       // stages 1 and 2 with fusion: the other tiles only
    nb.strips = bv.near_strips;
    nb.nstrips = bv.n_near_strips;
    for (int n = 0; n < steps; ++n) {
        for (int k = 1; k <= 4; ++k) {
            cudaError_t e = launch_ghost(bv, k, s);
            if (e != cudaSuccess) return e;
            const bool fused = bv.fuse12 && k <= 2;
            e = launch_stencil(fused ? nb : bv, k, ctas, s);
            if (e != cudaSuccess) return e;
            if (fused && k == 1 && (e = launch_pair(bv, s)) != cudaSuccess) return e;
        }
        cudaError_t e = launch_probes(bv, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Run `nsteps` steps, capturing 1-step and GRAPH_STEPS-step graphs on first use.
cudaError_t run_steps(const BatchView &bv, long long nsteps, cudaStream_t s, cudaGraphExec_t graph[2],
                      long long graph_launches[2]) {
    static const bool no_graph = getenv("LEE_NO_GRAPH") != nullptr;
    if (s == nullptr || no_graph) {
        while (nsteps > 0) {
            const int n = (int)std::min<long long>(nsteps, 1 << 20);
            cudaError_t e = enqueue_steps(bv, n, s);
            if (e != cudaSuccess) return e;
            nsteps -= n;
        }
        return cudaSuccess;
    }
    const int sizes[2] = {1, GRAPH_STEPS};
    for (int i = 0; i < 2; ++i) {
        if (graph[i]) continue;
        if (i == 1 && nsteps < GRAPH_STEPS) continue;
        cudaGraph_t gr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const long long before = launch_count();
        e = enqueue_steps(bv, sizes[i], s);
        graph_launches[i] = launch_count() - before;
        count_launch(-(int)graph_launches[i]);                  // replays are counted instead
        cudaError_t e2 = cudaStreamEndCapture(s, &gr);
        if (e != cudaSuccess) return e;
        if (e2 != cudaSuccess) return e2;
        e = cudaGraphInstantiate(&graph[i], gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return e;
    }
    while (nsteps >= GRAPH_STEPS && graph[1]) {
        cudaError_t e = cudaGraphLaunch(graph[1], s);
        if (e != cudaSuccess) return e;
        count_launch((int)graph_launches[1]);
        nsteps -= GRAPH_STEPS;
    }
    while (nsteps > 0) {
        cudaError_t e = cudaGraphLaunch(graph[0], s);
        if (e != cudaSuccess) return e;
        count_launch((int)graph_launches[0]);
        --nsteps;
    }
    return cudaSuccess;
}

BatchView single_view(lee_ctx *c) {
    BatchView bv{};
    bv.inst = c->dd;
    bv.ninst = 1;
    bv.tile_prefix = c->dprefix;
    bv.ghost_chunks = (const int4 *)(c->dev + c->L.chunks);
    bv.nchunks = n_chunks(c->hd.ng);
    bv.strips = (const int4 *)(c->dev + c->L.strips);
    bv.nstrips = c->nstrips;
    bv.use_tma = c->hd.use_tma;
    bv.kernel_mode = c->hd.kernel_mode;
    bv.tile_w = c->hd.tile_w;
    bv.tile_h = c->hd.tile_h;
    bv.band_chunks = (const int4 *)(c->dev + c->L.bchunks);
    bv.nband_chunks = c->nbchunks;
    bv.probe_inst = c->dprefix + 4;
    bv.nprobe_inst = c->hd.np > 0 ? 1 : 0;
    bv.total_tiles = c->hd.ntiles;
    bv.total_ghosts = c->hd.ng;
    bv.precision = c->g.precision;
    bv.ade_general = c->hd.ns != 2;
    bv.band_tile = default_band_tile_stages();
    return bv;
}

int reset_state(lee_ctx *ctx) {
    const Plan &P = ctx->plan;
    const size_t plane = (size_t)P.ny * P.pitch;
    CK(cudaMemsetAsync(ctx->dev + ctx->L.q, 0, 9 * plane * ctx->elem(), ctx->stream));
    const int ng = (int)P.g_target.size();
    if (ng) {
        CK(cudaMemsetAsync(ctx->dev + ctx->L.xn, 0, (size_t)ng * 8 * P.ns, ctx->stream));
        CK(cudaMemsetAsync(ctx->dev + ctx->L.xs, 0, (size_t)ng * 8 * P.ns, ctx->stream));
    }
    static const long long clk[8] = {-1, 0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(ctx->dev + ctx->L.clock, clk, sizeof clk, cudaMemcpyHostToDevice, ctx->stream));
    return LEE_OK;
}

}  // namespace

extern "C" {

const char *lee_version(void) { return "lee-b300 0.1 (sm_103a)"; }
long long lee_launch_count(void) { return launch_count(); }

int lee_create(lee_ctx **out, const lee_grid *g) {
    if (!out || !g) { g_create_err = "null argument"; return LEE_ERR_ARG; }
    const int minx = g->bc_x == LEE_BC_PERIODIC ? 7 : 8, miny = g->bc_y == LEE_BC_PERIODIC ? 7 : 8;
    if (g->nx < minx || g->ny < miny || !(g->h > 0) || !(g->cfl >= 0) ||
        (g->precision != LEE_FP64 && g->precision != LEE_FP32) ||
        (g->bc_x != LEE_BC_RADIATION && g->bc_x != LEE_BC_PERIODIC) ||
        (g->bc_y != LEE_BC_RADIATION && g->bc_y != LEE_BC_PERIODIC) ||
        (long long)g->nx * g->ny > (1LL << 31) / 4) {
        g_create_err = "invalid grid";
        return LEE_ERR_ARG;
    }
    lee_ctx *c = new lee_ctx();
    c->g = *g;
    *out = c;
    return LEE_OK;
}

int lee_destroy(lee_ctx *ctx) {
    if (!ctx) return LEE_ERR_ARG;
    drop_graphs(ctx->graph);
    delete ctx;
    return LEE_OK;
}

const char *lee_last_error(const lee_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int lee_set_wall_none(lee_ctx *ctx) {
    if (!ctx || ctx->planned) return ctx ? fail(ctx, LEE_ERR_ARG, "geometry is fixed after lee_plan") : LEE_ERR_ARG;
    ctx->geo = Geometry{};
    return LEE_OK;
}
int lee_set_wall_line(lee_ctx *ctx, double xw, double yw, double angle) {
    if (!ctx || ctx->planned) return ctx ? fail(ctx, LEE_ERR_ARG, "geometry is fixed after lee_plan") : LEE_ERR_ARG;
    if (!std::isfinite(xw) || !std::isfinite(yw) || !std::isfinite(angle)) return fail(ctx, LEE_ERR_ARG, "non-finite wall");
    ctx->geo = Geometry{1, xw, yw, angle};
    return LEE_OK;
}
int lee_set_wall_cylinder(lee_ctx *ctx, double xc, double yc, double r) {
    if (!ctx || ctx->planned) return ctx ? fail(ctx, LEE_ERR_ARG, "geometry is fixed after lee_plan") : LEE_ERR_ARG;
    if (!std::isfinite(xc) || !std::isfinite(yc) || !(r > 0)) return fail(ctx, LEE_ERR_ARG, "bad cylinder");
    ctx->geo = Geometry{2, xc, yc, r};
    return LEE_OK;
}
int lee_set_impedance(lee_ctx *ctx, double R, double M, double K) {
    if (!ctx || ctx->planned) return ctx ? fail(ctx, LEE_ERR_ARG, "impedance is fixed after lee_plan") : LEE_ERR_ARG;
    if (!(R > 0 && M > 0 && K > 0)) return fail(ctx, LEE_ERR_ARG, "impedance needs R, M, K > 0");
    ctx->imp = Impedance{false, R, M, K};
    return LEE_OK;
}
int lee_set_impedance_rational(lee_ctx *ctx, int n_real, const double *real, int n_pairs, const double *pairs) {
    if (!ctx || ctx->planned) return ctx ? fail(ctx, LEE_ERR_ARG, "impedance is fixed after lee_plan") : LEE_ERR_ARG;
    if (n_real < 0 || n_pairs < 0 || n_real + 2 * n_pairs < 1 || n_real + 2 * n_pairs > MAX_ADE_STATES ||
        (n_real && !real) || (n_pairs && !pairs))
        return fail(ctx, LEE_ERR_ARG, "rational admittance needs 1..8 states (n_real + 2 n_pairs)");
    Impedance imp;
    imp.rigid = false;
    imp.nreal = n_real;
    imp.npair = n_pairs;
    for (int k = 0; k < n_real; ++k) {
        imp.lam[k] = real[2 * k];
        imp.A[k] = real[2 * k + 1];
        if (!(imp.lam[k] < 0) || !std::isfinite(imp.A[k]))
            return fail(ctx, LEE_ERR_ARG, "rational admittance: real poles must be negative, residues finite");
    }
    for (int k = 0; k < n_pairs; ++k) {
        imp.al[k] = pairs[4 * k];
        imp.be[k] = pairs[4 * k + 1];
        imp.B[k] = pairs[4 * k + 2];
        imp.C[k] = pairs[4 * k + 3];
        if (!(imp.al[k] < 0 && imp.be[k] > 0) || !std::isfinite(imp.B[k]) || !std::isfinite(imp.C[k]))
            return fail(ctx, LEE_ERR_ARG, "rational admittance: pairs need alpha < 0 < beta, finite residues");
    }
    ctx->imp = imp;
    return LEE_OK;
}
int lee_set_rigid(lee_ctx *ctx) {
    if (!ctx || ctx->planned) return ctx ? fail(ctx, LEE_ERR_ARG, "impedance is fixed after lee_plan") : LEE_ERR_ARG;
    ctx->imp = Impedance{};
    return LEE_OK;
}

int lee_set_sponge(lee_ctx *ctx, int width, double kappa) {
    if (!ctx) return LEE_ERR_ARG;
    if (ctx->planned) return fail(ctx, LEE_ERR_ARG, "the absorbing ramp is fixed after lee_plan");
    if (width < 0 || (width > 0 && !(kappa >= 0.0 && std::isfinite(kappa))))
        return fail(ctx, LEE_ERR_ARG, "absorbing ramp needs width >= 0 and kappa >= 0");
    const int nmin = std::min(ctx->g.bc_x == LEE_BC_PERIODIC ? 1 << 30 : ctx->g.nx,
                              ctx->g.bc_y == LEE_BC_PERIODIC ? 1 << 30 : ctx->g.ny);
    if (width > 0 && 2 * width > nmin) return fail(ctx, LEE_ERR_ARG, "absorbing ramp wider than half the grid");
    ctx->sponge_w = width;
    ctx->sponge_k = width > 0 ? kappa : 0.0;
    return LEE_OK;
}

int lee_set_probes(lee_ctx *ctx, int n, const double *xy, int capacity) {
    if (!ctx) return LEE_ERR_ARG;
    if (ctx->planned) return fail(ctx, LEE_ERR_ARG, "probes are fixed after lee_plan");
    if (n < 0 || n > MAX_PROBES || (n > 0 && (!xy || capacity <= 0))) return fail(ctx, LEE_ERR_ARG, "bad probes");
    ctx->probe_xy.assign(xy, xy + 2 * n);
    ctx->probe_cap = n > 0 ? capacity : 0;
    return LEE_OK;
}

int lee_set_tile(lee_ctx *ctx, int tile_w, int tile_h) {
    if (!ctx) return LEE_ERR_ARG;
    if (ctx->planned) return fail(ctx, LEE_ERR_ARG, "the tile shape is fixed after lee_plan");
    if (tile_w == 0 && tile_h == 0) { ctx->tile_w_req = ctx->tile_h_req = 0; return LEE_OK; }
    const bool periodic = ctx->g.bc_x == LEE_BC_PERIODIC || ctx->g.bc_y == LEE_BC_PERIODIC;
    if (default_kernel_mode(ctx->g.precision, periodic) != KERNEL_TMA)
        return fail(ctx, LEE_ERR_ARG, "tile shapes are selectable for the FP32 TMA stencil only");
    if (!tma_tile_supported(tile_w, tile_h)) return fail(ctx, LEE_ERR_ARG, "unsupported tile shape");
    ctx->tile_w_req = tile_w;
    ctx->tile_h_req = tile_h;
    return LEE_OK;
}

int lee_plan(lee_ctx *ctx, lee_sizes *out) {
    if (!ctx || !out) return LEE_ERR_ARG;
    const lee_grid &g = ctx->g;
    std::string err;
    const bool periodic = g.bc_x == LEE_BC_PERIODIC || g.bc_y == LEE_BC_PERIODIC;
    ctx->kernel_mode = default_kernel_mode(g.precision, periodic);
    int tile_w = TILE_X, tile_h = TILE_Y;
    if (ctx->kernel_mode == KERNEL_TMA) {
        tma_tile(tile_w, tile_h);
        if (ctx->tile_w_req) { tile_w = ctx->tile_w_req; tile_h = ctx->tile_h_req; }
    }
    int rc = build_plan(g.nx, g.ny, g.h, g.x0, g.y0, g.bc_x == LEE_BC_PERIODIC, g.bc_y == LEE_BC_PERIODIC,
                        g.cfl * g.h, tile_w, tile_h, ctx->sponge_w, ctx->geo, ctx->imp, ctx->probe_xy, ctx->plan,
                        err);
    if (rc != LEE_OK) return fail(ctx, rc, err);
    if (ctx->plan.ade_amp > 1.0) {
        char b[160];
        snprintf(b, sizeof b, "ADE pole outside the RK4 region: max |P(pole dt)| = %.6g", ctx->plan.ade_amp);
        return fail(ctx, LEE_ERR_ADE_UNSTABLE, b);
    }
    ctx->L = make_layout(ctx);
    ctx->planned = true;
    std::memset(out, 0, sizeof *out);
    out->device_bytes = (long long)ctx->L.total;
    out->n_ghost = (int)ctx->plan.g_target.size();
    out->n_fluid = ctx->plan.n_fluid;
    out->n_entries = (long long)ctx->plan.e_idx.size();
    out->n_reduced = ctx->plan.n_reduced;
    out->regime = ctx->plan.regime;
    out->dt = g.cfl * g.h;
    out->ade_amplification = ctx->plan.ade_amp;
    out->n_tiles = ctx->plan.tiles_x * ctx->plan.tiles_y;
    out->n_states = ctx->plan.ns;
    return LEE_OK;
}

int lee_bind(lee_ctx *ctx, void *dev_ptr, long long dev_bytes, void *stream) {
    if (!ctx) return LEE_ERR_ARG;
    if (!ctx->planned) return fail(ctx, LEE_ERR_ARG, "lee_bind before lee_plan");
    if (!dev_ptr || ((uintptr_t)dev_ptr % ALIGN) != 0) return fail(ctx, LEE_ERR_ARG, "device pointer must be 256-byte aligned");
    if (dev_bytes < (long long)ctx->L.total) return fail(ctx, LEE_ERR_BUDGET, "device buffer smaller than lee_plan's device_bytes");
    drop_graphs(ctx->graph);
    ctx->dev = (char *)dev_ptr;
    ctx->stream = (cudaStream_t)stream;
    const Plan &P = ctx->plan;
    const Layout &L = ctx->L;
    const int ng = (int)P.g_target.size();
    const size_t plane = (size_t)P.ny * P.pitch;
    cudaStream_t s = ctx->stream;
    // FP32 bulk: weights as float-float pairs for the FP32-pipe ghost gather
    std::vector<GWF> wff;
    if (ghost_float_float(ctx->g.precision)) {
        wff.resize(P.e_w.size() / 4);
        for (size_t e = 0; e < wff.size(); ++e)
            for (int r = 0; r < 4; ++r) {
                const double w = P.e_w[4 * e + r];
                const float hi = (float)w;
                if (!std::isfinite(hi)) return fail(ctx, LEE_ERR_GEOMETRY, "ghost weight outside the FP32 range");
                wff[e].hi[r] = hi;
                wff[e].lo[r] = (float)(w - (double)hi);     // w - hi is exact in FP64
            }
    }
    CK(prepare_kernels(ctx->g.precision));
    CK(cudaMemsetAsync(ctx->dev, 0, L.total, s));
    std::vector<int4> chunks;                 // ghost work list (after the memset above)
    append_chunks(chunks, 0, ng);
    if (!chunks.empty())
        CK(cudaMemcpyAsync(ctx->dev + L.chunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    // mask in pitch layout
    std::vector<uint8_t> mask(plane, 0);
    for (int j = 0; j < P.ny; ++j) std::memcpy(&mask[(size_t)j * P.pitch], &P.kind[(size_t)j * P.nx], P.nx);
    auto to_pitch = [&](int idx) { return (idx / P.nx) * P.pitch + idx % P.nx; };
    std::vector<int> gt(ng), ei(P.e_idx.size()), pidx(P.p_idx.size());
    for (int q = 0; q < ng; ++q) gt[q] = to_pitch(P.g_target[q]);
    for (size_t e = 0; e < ei.size(); ++e) ei[e] = to_pitch(P.e_idx[e]);
    for (size_t e = 0; e < pidx.size(); ++e) pidx[e] = to_pitch(P.p_idx[e]);
    std::vector<double> gn((size_t)2 * ng);
    for (int q = 0; q < ng; ++q) { gn[2 * q] = P.g_meta[5 * q + 2]; gn[2 * q + 1] = P.g_meta[5 * q + 3]; }
    CK(cudaMemcpyAsync(ctx->dev + L.mask, mask.data(), plane, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->dev + L.tiles, P.tile_flags.data(), P.tile_flags.size() * 4, cudaMemcpyHostToDevice, s));
    if (ng) {
        CK(cudaMemcpyAsync(ctx->dev + L.gt, gt.data(), (size_t)ng * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->dev + L.gs, P.g_start.data(), (size_t)(ng + 1) * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->dev + L.gn, gn.data(), (size_t)ng * 16, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->dev + L.gk, P.g_kappa.data(), (size_t)ng * 16, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->dev + L.ei, ei.data(), ei.size() * 4, cudaMemcpyHostToDevice, s));
        if (!wff.empty())
            CK(cudaMemcpyAsync(ctx->dev + L.ew, wff.data(), wff.size() * sizeof(GWF), cudaMemcpyHostToDevice, s));
        else
            CK(cudaMemcpyAsync(ctx->dev + L.ew, P.e_w.data(), P.e_w.size() * 8, cudaMemcpyHostToDevice, s));
    }
    if (!P.ade_coef.empty())
        CK(cudaMemcpyAsync(ctx->dev + L.ade, P.ade_coef.data(), P.ade_coef.size() * 8, cudaMemcpyHostToDevice, s));
    const int np = (int)ctx->probe_xy.size() / 2;
    if (np) {
        CK(cudaMemcpyAsync(ctx->dev + L.pi, pidx.data(), pidx.size() * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(ctx->dev + L.pw, P.p_w.data(), P.p_w.size() * 8, cudaMemcpyHostToDevice, s));
    }
    // [0..1] tile prefix, [2..3] ghost prefix, [4] probe instance
    ctx->nband = ctx_band_nodes(ctx);
    std::vector<int4> bch;
    band_chunks(0, ctx->nband, bch, P.kind.data(), P.nx, P.ny);
    ctx->nbchunks = (int)bch.size();
    if (!bch.empty())
        CK(cudaMemcpyAsync(ctx->dev + L.bchunks, bch.data(), bch.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    const int prefix[8] = {0, P.tiles_x * P.tiles_y, 0, ng, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(ctx->dev + L.prefix, prefix, sizeof prefix, cudaMemcpyHostToDevice, s));
    InstDesc &d = ctx->hd;
    d = InstDesc{};
    for (int b = 0; b < 3; ++b) d.q[b] = ctx->dev + L.q + (size_t)b * 3 * plane * ctx->elem();
    d.plane = (long long)plane;
    d.mask = (const uint8_t *)(ctx->dev + L.mask);
    d.tile_flags = (const uint32_t *)(ctx->dev + L.tiles);
    d.nx = P.nx; d.ny = P.ny; d.pitch = P.pitch; d.tiles_x = P.tiles_x; d.tiles_y = P.tiles_y;
    d.ntiles = P.tiles_x * P.tiles_y;
    d.tile_h = P.tile_h;
    d.tile_w = P.tile_w;
    d.per_x = ctx->g.bc_x == LEE_BC_PERIODIC; d.per_y = ctx->g.bc_y == LEE_BC_PERIODIC;
    d.h = ctx->g.h; d.inv_h = 1.0 / ctx->g.h; d.dt = ctx->g.cfl * ctx->g.h;
    fill_stage_constants(d.dt, d.h, ctx->sponge_k, d.kf, d.kd);
    d.sponge_w = ctx->sponge_w;
    d.cx = 0.5 * (P.nx - 1); d.cy = 0.5 * (P.ny - 1);
    d.ng = ng;
    d.g_target = (const int *)(ctx->dev + L.gt);
    d.g_start = (const int *)(ctx->dev + L.gs);
    d.g_n = (const double2 *)(ctx->dev + L.gn);
    d.g_kappa = (const double2 *)(ctx->dev + L.gk);
    d.e_idx = (const int *)(ctx->dev + L.ei);
    d.e_w = (const GW *)(ctx->dev + L.ew);
    d.Xn = (double *)(ctx->dev + L.xn);
    d.Xs = (double *)(ctx->dev + L.xs);
    for (int q = 0; q < 4; ++q) d.A[q] = P.A[q];
    d.b[0] = P.b[0]; d.b[1] = P.b[1]; d.c[0] = P.c[0]; d.c[1] = P.c[1];
    d.gx = ctx->dev + L.gx;
    d.gy = ctx->dev + L.gy;
    d.np = np; d.pcap = ctx->probe_cap;
    d.p_idx = (const int *)(ctx->dev + L.pi);
    d.p_w = (const double *)(ctx->dev + L.pw);
    d.p_hist = (double *)(ctx->dev + L.ph);
    d.clock = (long long *)(ctx->dev + L.clock);
    d.scratch = (double *)(ctx->dev + L.scratch);
    d.staging = (double *)(ctx->dev + L.staging);
    d.bc = (const double *)(ctx->dev + L.bc);
    d.ade = (const double *)(ctx->dev + L.ade);
    d.ns = P.ns;
    d.precision = ctx->g.precision;
    d.kernel_mode = ctx->kernel_mode;
    d.use_tma = ctx->kernel_mode == KERNEL_TMA;
    {
        std::vector<int4> strips;
        append_strips(strips, 0, d, strip_segment((long long)d.tiles_x * d.tiles_y), P.tile_flags);
        ctx->nstrips = (int)strips.size();
        CK(cudaMemcpyAsync(ctx->dev + L.strips, strips.data(), strips.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    for (int q = 0; q < 4; ++q) d.tmap[q] = ctx->dev + L.tmap + 128 * q;
    if (d.use_tma) {
        alignas(64) unsigned char maps[4 * 128];
        std::string terr;
        if (!encode_tensor_maps(d, maps, terr)) return fail(ctx, LEE_ERR_CUDA, "tensor map: " + terr);
        CK(cudaMemcpyAsync(ctx->dev + L.tmap, maps, sizeof maps, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    ctx->dd = (InstDesc *)(ctx->dev + L.desc);
    ctx->dprefix = (int *)(ctx->dev + L.prefix);
    ctx->bound = true;
    int rc = upload_source(ctx);          // also uploads the descriptor and synchronises
    if (rc != LEE_OK) { ctx->bound = false; return rc; }
    rc = reset_state(ctx);
    if (rc != LEE_OK) return rc;
    CK(cudaStreamSynchronize(s));
    return LEE_OK;
}

int lee_set_monopole(lee_ctx *ctx, double xs, double ys, double amp, double halfwidth, double omega) {
    if (!ctx) return LEE_ERR_ARG;
    if (!(halfwidth > 0) || !std::isfinite(amp) || !std::isfinite(omega) || !std::isfinite(xs) || !std::isfinite(ys))
        return fail(ctx, LEE_ERR_ARG, "bad monopole");
    if (std::fabs(omega * ctx->g.cfl * ctx->g.h) > 10.0) return fail(ctx, LEE_ERR_ARG, "source period shorter than 0.6 steps");
    ctx->s_xs = xs; ctx->s_ys = ys; ctx->s_amp = amp; ctx->s_w = halfwidth; ctx->s_omega = omega;
    if (ctx->bound) return upload_source(ctx);
    return LEE_OK;
}

static int init_common(lee_ctx *ctx, int kind, const double *prm) {
    if (!ctx) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "init before lee_bind");
    int rc = reset_state(ctx);
    if (rc != LEE_OK) return rc;
    CK(launch_init(ctx->dd, ctx->hd, kind, prm, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

int lee_init_pulse(lee_ctx *ctx, double xs, double ys, double amp, double halfwidth) {
    if (ctx && !(halfwidth > 0)) return fail(ctx, LEE_ERR_ARG, "halfwidth must be > 0");
    const double prm[8] = {xs, ys, amp, std::log(2.0) / (halfwidth * halfwidth), 0, 0,
                           ctx ? ctx->g.x0 : 0, ctx ? ctx->g.y0 : 0};
    return init_common(ctx, 0, prm);
}

int lee_init_packet(lee_ctx *ctx, double xs, double ys, double angle, double amp, double k, double alpha) {
    const double prm[8] = {xs, ys, angle, amp, k, alpha, ctx ? ctx->g.x0 : 0, ctx ? ctx->g.y0 : 0};
    return init_common(ctx, 1, prm);
}

int lee_write_field(lee_ctx *ctx, int which, const double *host) {
    if (!ctx || !host || which < 0 || which > 2) return ctx ? fail(ctx, LEE_ERR_ARG, "bad field") : LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    CK(cudaMemcpyAsync(ctx->hd.staging, host, (size_t)ctx->g.nx * ctx->g.ny * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_from_staging(ctx->dd, ctx->hd, which, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

int lee_step(lee_ctx *ctx, long long nsteps) {
    if (!ctx) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "lee_step before lee_bind");
    if (nsteps < 0) return fail(ctx, LEE_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return LEE_OK;
    CK(run_steps(single_view(ctx), nsteps, ctx->stream, ctx->graph, ctx->graph_launches));
    return LEE_OK;
}

int lee_sync(lee_ctx *ctx) {
    if (!ctx) return LEE_ERR_ARG;
    if (!ctx->bound) return LEE_OK;
    long long st = 0;
    CK(cudaMemcpyAsync(&st, ctx->hd.clock + 2, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st & (long long)STATUS_TIMEOUT) return fail(ctx, LEE_ERR_TIMEOUT, "a stencil kernel gave up waiting for a tile copy");
    if (st & (long long)STATUS_DIVERGED) return fail(ctx, LEE_ERR_DIVERGED, "a ghost, ADE or probe value is not finite");
    return LEE_OK;
}

int lee_read_field(lee_ctx *ctx, int which, double *host) {
    if (!ctx || !host || which < 0 || which > 2) return ctx ? fail(ctx, LEE_ERR_ARG, "bad field") : LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    CK(launch_to_staging(ctx->dd, ctx->hd, which, 0, ctx->stream));
    CK(cudaMemcpyAsync(host, ctx->hd.staging, (size_t)ctx->g.nx * ctx->g.ny * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

int lee_read_mask(lee_ctx *ctx, unsigned char *host) {
    if (!ctx || !host) return LEE_ERR_ARG;
    if (!ctx->planned) return fail(ctx, LEE_ERR_ARG, "not planned");
    std::memcpy(host, ctx->plan.kind.data(), ctx->plan.kind.size());
    return LEE_OK;
}

int lee_tile_flags(lee_ctx *ctx, unsigned int *host, int *tiles_x, int *tiles_y) {
    if (!ctx || !tiles_x || !tiles_y) return LEE_ERR_ARG;
    if (!ctx->planned) return fail(ctx, LEE_ERR_ARG, "not planned");
    *tiles_x = ctx->plan.tiles_x;
    *tiles_y = ctx->plan.tiles_y;
    if (host) std::memcpy(host, ctx->plan.tile_flags.data(), ctx->plan.tile_flags.size() * sizeof(unsigned int));
    return LEE_OK;
}

int lee_read_ade(lee_ctx *ctx, double *host) {
    if (!ctx || !host) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    if (ctx->hd.ng == 0) return LEE_OK;
    CK(cudaMemcpyAsync(host, ctx->hd.Xn, (size_t)ctx->hd.ng * 8 * ctx->hd.ns, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

int lee_get_step(lee_ctx *ctx, long long *steps) {
    if (!ctx || !steps) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    long long clk[2];
    CK(cudaMemcpyAsync(clk, ctx->hd.clock, sizeof clk, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *steps = clk[0] + 1;
    return LEE_OK;
}

int lee_read_probes(lee_ctx *ctx, double *host, long long *nrec) {
    if (!ctx || !nrec) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    long long clk[2];
    CK(cudaMemcpyAsync(clk, ctx->hd.clock, sizeof clk, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *nrec = clk[1];
    if (host && clk[1] > 0 && ctx->hd.np > 0) {
        CK(cudaMemcpyAsync(host, ctx->hd.p_hist, (size_t)clk[1] * ctx->hd.np * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return LEE_OK;
}

int lee_energy(lee_ctx *ctx, double *out) {
    if (!ctx || !out) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    CK(cudaMemsetAsync(ctx->hd.scratch, 0, 8, ctx->stream));
    CK(launch_energy(ctx->dd, ctx->hd, ctx->stream));
    double e = 0;
    CK(cudaMemcpyAsync(&e, ctx->hd.scratch, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out = 0.5 * ctx->g.h * ctx->g.h * e;
    return LEE_OK;
}

// state blob: clock[2] | Q^n (3 planes, bulk precision) | X^n | probe history
int lee_state_bytes(lee_ctx *ctx, long long *bytes) {
    if (!ctx || !bytes) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    *bytes = 16 + 3 * ctx->hd.plane * (long long)ctx->elem() + 8LL * ctx->hd.ns * ctx->hd.ng +
             8LL * ctx->hd.np * ctx->hd.pcap;
    return LEE_OK;
}

int lee_read_state(lee_ctx *ctx, void *blob) {
    long long nb;
    int rc = lee_state_bytes(ctx, &nb);
    if (rc != LEE_OK) return rc;
    char *b = (char *)blob;
    const size_t qb = 3 * (size_t)ctx->hd.plane * ctx->elem();
    CK(cudaMemcpyAsync(b, ctx->hd.clock, 16, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(b + 16, ctx->hd.q[0], qb, cudaMemcpyDeviceToHost, ctx->stream));
    const size_t xb = 8 * (size_t)ctx->hd.ns * ctx->hd.ng;
    if (ctx->hd.ng) CK(cudaMemcpyAsync(b + 16 + qb, ctx->hd.Xn, xb, cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->hd.np) CK(cudaMemcpyAsync(b + 16 + qb + xb, ctx->hd.p_hist,
                                       8 * (size_t)ctx->hd.np * ctx->hd.pcap, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

int lee_write_state(lee_ctx *ctx, const void *blob) {
    long long nb;
    int rc = lee_state_bytes(ctx, &nb);
    if (rc != LEE_OK) return rc;
    const char *b = (const char *)blob;
    const size_t qb = 3 * (size_t)ctx->hd.plane * ctx->elem();
    CK(cudaMemcpyAsync(ctx->hd.clock, b, 16, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->hd.clock + 2, 0, sizeof(long long), ctx->stream));   // status: healthy
    CK(cudaMemcpyAsync(ctx->hd.q[0], b + 16, qb, cudaMemcpyHostToDevice, ctx->stream));
    const size_t xb = 8 * (size_t)ctx->hd.ns * ctx->hd.ng;
    // X^n only: stage 1 reads the step's starting ADE state from X^n
    if (ctx->hd.ng) CK(cudaMemcpyAsync(ctx->hd.Xn, b + 16 + qb, xb, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->hd.np) CK(cudaMemcpyAsync(ctx->hd.p_hist, b + 16 + qb + xb,
                                       8 * (size_t)ctx->hd.np * ctx->hd.pcap, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

int lee_upload_state_async(lee_ctx *ctx, const void *blob) {
    long long nb;
    int rc = lee_state_bytes(ctx, &nb);
    if (rc != LEE_OK) return rc;
    const char *b = (const char *)blob;
    const size_t qb = 3 * (size_t)ctx->hd.plane * ctx->elem();
    CK(cudaMemcpyAsync(ctx->hd.clock, b, 16, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(ctx->hd.clock + 2, 0, sizeof(long long), ctx->stream));   // status: healthy
    CK(cudaMemcpyAsync(ctx->hd.q[0], b + 16, qb, cudaMemcpyHostToDevice, ctx->stream));
    const size_t xb = 8 * (size_t)ctx->hd.ns * ctx->hd.ng;
    // X^n only: stage 1 reads the step's starting ADE state from X^n
    if (ctx->hd.ng) CK(cudaMemcpyAsync(ctx->hd.Xn, b + 16 + qb, xb, cudaMemcpyHostToDevice, ctx->stream));
    return LEE_OK;
}

int lee_download_probes_async(lee_ctx *ctx, double *host, long long first, long long count) {
    if (!ctx || !host || first < 0 || count < 0) return ctx ? fail(ctx, LEE_ERR_ARG, "bad probe range") : LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "not bound");
    if (first + count > ctx->hd.pcap) return fail(ctx, LEE_ERR_ARG, "probe range beyond capacity");
    if (count == 0 || ctx->hd.np == 0) return LEE_OK;
    CK(cudaMemcpyAsync(host, ctx->hd.p_hist + first * ctx->hd.np, (size_t)count * ctx->hd.np * 8,
                       cudaMemcpyDeviceToHost, ctx->stream));
    return LEE_OK;
}

int lee_ghost_info(lee_ctx *ctx, int g, int *target, double *meta, int *m, int *ncloud) {
    if (!ctx) return LEE_ERR_ARG;
    if (!ctx->planned) return fail(ctx, LEE_ERR_ARG, "not planned");
    const Plan &P = ctx->plan;
    if (g < 0 || g >= (int)P.g_target.size()) return fail(ctx, LEE_ERR_ARG, "ghost index out of range");
    if (target) *target = P.g_target[g];
    if (meta) for (int q = 0; q < 5; ++q) meta[q] = P.g_meta[5 * g + q];
    if (m) *m = P.g_m[g];
    if (ncloud) *ncloud = P.g_start[g + 1] - P.g_start[g];
    return LEE_OK;
}

int lee_ghost_weights(lee_ctx *ctx, int g, int *idx, double *w, double *kappa) {
    if (!ctx) return LEE_ERR_ARG;
    if (!ctx->planned) return fail(ctx, LEE_ERR_ARG, "not planned");
    const Plan &P = ctx->plan;
    if (g < 0 || g >= (int)P.g_target.size()) return fail(ctx, LEE_ERR_ARG, "ghost index out of range");
    const int a = P.g_start[g], b = P.g_start[g + 1];
    for (int e = a; e < b; ++e) {
        if (idx) idx[e - a] = P.e_idx[e];
        if (w) for (int q = 0; q < 4; ++q) w[4 * (e - a) + q] = P.e_w[4 * (size_t)e + q];
    }
    if (kappa) { kappa[0] = P.g_kappa[2 * g]; kappa[1] = P.g_kappa[2 * g + 1]; }
    return LEE_OK;
}

int lee_fill_ghosts_with_bc(lee_ctx *ctx, const double *bc) {
    if (!ctx) return LEE_ERR_ARG;
    if (!ctx->bound) return fail(ctx, LEE_ERR_ARG, "lee_fill_ghosts_with_bc before lee_bind");
    const int ng = (int)ctx->plan.g_target.size();
    if (ng == 0) return LEE_OK;
    if (!bc) return fail(ctx, LEE_ERR_ARG, "null boundary data");
    CK(cudaMemcpyAsync(ctx->dev + ctx->L.bc, bc, (size_t)ng * 16, cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_ghost(single_view(ctx), 0, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return LEE_OK;
}

// ------------------------------------------------------------------ batches
int lee_batch_create(lee_batch **out, int precision) {
    if (!out || (precision != LEE_FP32 && precision != LEE_FP64)) return LEE_ERR_ARG;
    lee_batch *b = new lee_batch();
    b->precision = precision;
    *out = b;
    return LEE_OK;
}

int lee_batch_destroy(lee_batch *b) {
    if (!b) return LEE_ERR_ARG;
    drop_graphs(b->graph);
    delete b;
    return LEE_OK;
}

const char *lee_batch_last_error(const lee_batch *b) { return b ? b->err.c_str() : ""; }

int lee_batch_add(lee_batch *b, lee_ctx *c) {
    if (!b || !c) return LEE_ERR_ARG;
    if (!c->bound) { b->err = "context not bound"; return LEE_ERR_ARG; }
    if (c->g.precision != b->precision) { b->err = "precision differs from the batch"; return LEE_ERR_ARG; }
    if (!b->members.empty() && (b->members[0]->hd.kernel_mode != c->hd.kernel_mode ||
                                b->members[0]->hd.tile_w != c->hd.tile_w ||
                                b->members[0]->hd.tile_h != c->hd.tile_h)) {
        b->err = "members use different stencil kernels (periodic axes or kernel selection): batch them separately";
        return LEE_ERR_ARG;
    }
    if (std::find(b->members.begin(), b->members.end(), c) != b->members.end()) { b->err = "already a member"; return LEE_ERR_ARG; }
    b->members.push_back(c);
    b->dirty = true;
    return LEE_OK;
}

int lee_batch_remove(lee_batch *b, lee_ctx *c) {
    if (!b || !c) return LEE_ERR_ARG;
    auto it = std::find(b->members.begin(), b->members.end(), c);
    if (it == b->members.end()) { b->err = "not a member"; return LEE_ERR_ARG; }
    b->members.erase(it);
    b->dirty = true;
    return LEE_OK;
}

static long long batch_bytes(const lee_batch *b) {
    const size_t n = std::max<size_t>(b->members.size(), 1);
    size_t nch = 1, nst = 1, nbc = 1;
    for (auto *c : b->members) {
        nch += n_chunks(c->hd.ng);
        nst += (size_t)c->hd.tiles_x * c->hd.tiles_y;
        nbc += c->nbchunks;
    }
    size_t npv = 1;
    for (auto *c : b->members) npv += c->hd.np;
    return (long long)(align_up(n * sizeof(InstDesc)) + 2 * align_up((n + 1) * 4) + align_up(nch * sizeof(int4)) +
                       3 * align_up(nst * sizeof(int4)) + align_up(n * sizeof(long long)) + align_up(nbc * sizeof(int4)) +
                       align_up((n + 1) * 4) + align_up(npv * 8));
}

int lee_batch_plan(lee_batch *b, long long *device_bytes) {
    if (!b || !device_bytes) return LEE_ERR_ARG;
    *device_bytes = batch_bytes(b);
    return LEE_OK;
}

int lee_batch_bind(lee_batch *b, void *dev_ptr, long long dev_bytes, void *stream) {
    if (!b || !dev_ptr || ((uintptr_t)dev_ptr % ALIGN)) return LEE_ERR_ARG;
    b->dev = (char *)dev_ptr;
    b->bytes = dev_bytes;
    b->stream = (cudaStream_t)stream;
    b->dirty = true;
    return LEE_OK;
}

static int batch_refresh(lee_batch *b) {
    const size_t n = b->members.size();
    if (batch_bytes(b) > b->bytes) { b->err = "batch buffer too small"; return LEE_ERR_BUDGET; }
    std::vector<InstDesc> descs(n);
    std::vector<int> tp(n + 1, 0), pi;
    std::vector<int4> bch;
    std::vector<int4> chunks, strips;
    int total_ghosts = 0;
    long long total_tiles = 0;
    for (auto *c : b->members) total_tiles += c->hd.ntiles;
    const int seg = strip_segment(total_tiles, b->strips_per_sm);
    for (size_t i = 0; i < n; ++i) {
        descs[i] = b->members[i]->hd;
        tp[i + 1] = tp[i] + descs[i].ntiles;
        band_chunks((int)i, b->members[i]->nband, bch, b->members[i]->plan.kind.data(), b->members[i]->plan.nx,
                    b->members[i]->plan.ny);
        append_chunks(chunks, (int)i, descs[i].ng);
        append_strips(strips, (int)i, descs[i], seg, b->members[i]->plan.tile_flags);
        total_ghosts += descs[i].ng;
        if (descs[i].np > 0) pi.push_back((int)i);
    }
    pi.resize(std::max<size_t>(pi.size(), 1));
    chunks.resize(std::max<size_t>(chunks.size(), 1));
    sort_strips(strips);
    const int nstrips = (int)strips.size();
    strips.resize(std::max<size_t>(strips.size(), 1));
    // fused stages 1 + 2: the tiles clear of walls, band and ramp, and strips of the others
    std::vector<int4> far, near;
    bool fuse = b->fuse12 != 0 && n > 0;
    for (size_t i = 0; fuse && i < n; ++i)
        fuse = descs[i].precision == LEE_FP32 && descs[i].kernel_mode == KERNEL_TMA && b->members[i]->nband > 0 &&
               descs[i].tile_w == pair_tile_w() && descs[i].tile_h == pair_tile_h();
    if (fuse) {
        for (size_t i = 0; i < n; ++i) {
            const lee_ctx *c = b->members[i];
            const InstDesc &d = descs[i];
            const int m = std::max(3, d.sponge_w);
            std::vector<char> isfar((size_t)d.tiles_x * d.tiles_y, 0);
            for (int ty = 0; ty < d.tiles_y; ++ty)
                for (int tx = 0; tx < d.tiles_x; ++tx) {
                    const int x0 = tx * d.tile_w, y0 = ty * d.tile_h;
                    bool ok = c->s_amp == 0.0 && x0 - 8 >= 0 && y0 - 8 >= 0 && x0 + d.tile_w + 7 <= d.nx - 1 &&
                              y0 + d.tile_h + 7 <= d.ny - 1 && x0 - 3 >= m && y0 - 3 >= m &&
                              x0 + d.tile_w + 2 <= d.nx - 1 - m && y0 + d.tile_h + 2 <= d.ny - 1 - m;
                    for (int y = y0 - 3; ok && y <= y0 + d.tile_h + 2; ++y)
                        for (int x = x0 - 3; x <= x0 + d.tile_w + 2; ++x)
                            if (c->plan.kind[(size_t)y * d.nx + x] != 1) { ok = false; break; }
                    if (ok) { isfar[(size_t)ty * d.tiles_x + tx] = 1; far.push_back(make_int4((int)i, x0, y0, 0)); }
                }
            const std::vector<uint32_t> &tf = c->plan.tile_flags;
            auto skip = [&](int tx, int ty) {
                const size_t t = (size_t)ty * d.tiles_x + tx;
                return isfar[t] || (tf[t] & TILE_INERT);
            };
            for (int tx = 0; tx < d.tiles_x; ++tx)
                for (int ty = 0; ty < d.tiles_y;) {
                    if (skip(tx, ty)) { ++ty; continue; }
                    int len = 0;
                    while (ty + len < d.tiles_y && !skip(tx, ty + len) && len < seg) ++len;
                    near.push_back(make_int4((int)i, tx, ty, len));
                    ty += len;
                }
        }
        sort_strips(near);
    }
    const int nnear = (int)near.size(), nfar = (int)far.size();
    near.resize(std::max<size_t>(near.size(), 1));
    far.resize(std::max<size_t>(far.size(), 1));
    const size_t o_desc = 0, o_tp = align_up(n * sizeof(InstDesc)), o_pi = o_tp + align_up((n + 1) * 4),
                 o_ch = o_pi + align_up((n + 1) * 4), o_st = o_ch + align_up(chunks.size() * sizeof(int4)),
                 o_near = o_st + align_up(strips.size() * sizeof(int4)),
                 o_far = o_near + align_up(near.size() * sizeof(int4)),
                 o_status = o_far + align_up(far.size() * sizeof(int4)),
                 o_bc = o_status + align_up(n * sizeof(long long));
    b->status = (long long *)(b->dev + o_status);
    // the members' latest probe records side by side (lee_batch_read_latest_probes_async)
    std::vector<int> poff(pi.size() + 1, 0);
    for (size_t i = 0; i < pi.size(); ++i) poff[i + 1] = poff[i] + (n ? descs[pi[i]].np : 0);
    const size_t o_poff = o_bc + align_up(std::max<size_t>(bch.size(), 1) * sizeof(int4)),
                 o_pbuf = o_poff + align_up((n + 1) * 4);
    b->probe_off = (int *)(b->dev + o_poff);
    b->probe_buf = (double *)(b->dev + o_pbuf);
    b->nprobe_values = poff.back();
    cudaError_t e;
    if (n) {
        if ((e = cudaMemcpyAsync(b->dev + o_desc, descs.data(), n * sizeof(InstDesc), cudaMemcpyHostToDevice, b->stream)) ||
            (e = cudaMemcpyAsync(b->dev + o_tp, tp.data(), (n + 1) * 4, cudaMemcpyHostToDevice, b->stream)) ||
            (e = cudaMemcpyAsync(b->dev + o_pi, pi.data(), pi.size() * 4, cudaMemcpyHostToDevice, b->stream)) ||
            (e = cudaMemcpyAsync(b->dev + o_ch, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream)) ||
            (e = cudaMemcpyAsync(b->dev + o_st, strips.data(), strips.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream)) ||
            (e = cudaMemcpyAsync(b->dev + o_near, near.data(), near.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream)) ||
            (e = cudaMemcpyAsync(b->dev + o_far, far.data(), far.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream)) ||
            (bch.size() && (e = cudaMemcpyAsync(b->dev + o_bc, bch.data(), bch.size() * sizeof(int4),
                                                cudaMemcpyHostToDevice, b->stream))) ||
            (e = cudaMemcpyAsync(b->dev + o_poff, poff.data(), poff.size() * 4, cudaMemcpyHostToDevice, b->stream)) ||
            (e = cudaStreamSynchronize(b->stream))) {
            b->err = std::string("batch upload: ") + cudaGetErrorString(e);
            return LEE_ERR_CUDA;
        }
    }
    BatchView &bv = b->bv;
    bv.inst = (const InstDesc *)(b->dev + o_desc);
    bv.ninst = (int)n;
    bv.tile_prefix = (const int *)(b->dev + o_tp);
    bv.ghost_chunks = (const int4 *)(b->dev + o_ch);
    bv.nchunks = total_ghosts > 0 ? (int)chunks.size() : 0;
    bv.strips = (const int4 *)(b->dev + o_st);
    bv.nstrips = nstrips;
    bv.use_tma = n ? descs[0].use_tma : 0;
    bv.kernel_mode = n ? descs[0].kernel_mode : KERNEL_SMEM;
    bv.tile_w = n ? descs[0].tile_w : TILE_X;
    bv.tile_h = n ? descs[0].tile_h : TILE_Y;
    bv.band_chunks = (const int4 *)(b->dev + o_bc);
    bv.nband_chunks = (int)bch.size();
    bv.probe_inst = (const int *)(b->dev + o_pi);
    bv.nprobe_inst = 0;
    for (auto *c : b->members) bv.nprobe_inst += c->hd.np > 0;
    bv.total_tiles = tp[n];
    bv.total_ghosts = total_ghosts;
    bv.precision = b->precision;
    bv.ade_general = 0;
    for (size_t i = 0; i < n; ++i) bv.ade_general |= descs[i].ns != 2;
    bv.fuse12 = fuse && nfar > 0;
    bv.band_tile = b->band_tile < 0 ? default_band_tile_stages() : b->band_tile;
    bv.near_strips = (const int4 *)(b->dev + o_near);
    bv.n_near_strips = nnear;
    bv.far_tiles = (const int4 *)(b->dev + o_far);
    bv.n_far_tiles = nfar;
    drop_graphs(b->graph);
    b->dirty = false;
    return LEE_OK;
}

int lee_batch_step(lee_batch *b, long long nsteps) {
    if (!b) return LEE_ERR_ARG;
    if (!b->dev) { b->err = "batch not bound"; return LEE_ERR_ARG; }
    if (b->dirty) {
        int rc = batch_refresh(b);
        if (rc != LEE_OK) return rc;
    }
    if (b->members.empty() || nsteps <= 0) return LEE_OK;
    cudaError_t e = run_steps(b->bv, nsteps, b->stream, b->graph, b->graph_launches);
    if (e != cudaSuccess) { b->err = std::string("batch step: ") + cudaGetErrorString(e); return LEE_ERR_CUDA; }
    return LEE_OK;
}

int lee_batch_status(lee_batch *b, long long *host, int n) {
    if (!b || (n > 0 && !host)) return LEE_ERR_ARG;
    if (!b->dev) { b->err = "batch not bound"; return LEE_ERR_ARG; }
    if (n != (int)b->members.size()) { b->err = "n differs from the member count"; return LEE_ERR_ARG; }
    if (b->dirty) {
        int rc = batch_refresh(b);
        if (rc != LEE_OK) return rc;
    }
    if (n == 0) return LEE_OK;
    cudaError_t e;
    if ((e = launch_status_gather(b->bv, b->status, b->stream)) ||
        (e = cudaMemcpyAsync(host, b->status, (size_t)n * sizeof(long long), cudaMemcpyDeviceToHost, b->stream)) ||
        (e = cudaStreamSynchronize(b->stream))) {
        b->err = std::string("batch status: ") + cudaGetErrorString(e);
        return LEE_ERR_CUDA;
    }
    return LEE_OK;
}

int lee_batch_set_stage_fusion(lee_batch *b, int on) {
    if (!b) return LEE_ERR_ARG;
    b->fuse12 = on != 0;
    b->dirty = true;
    return LEE_OK;
}

int lee_batch_set_band_in_tile(lee_batch *b, int stage_mask) {
    if (!b || stage_mask < -1 || (stage_mask > 0 && (stage_mask & ~28))) return LEE_ERR_ARG;
    b->band_tile = stage_mask;
    b->dirty = true;
    return LEE_OK;
}

int lee_batch_band_in_tile(lee_batch *b, int *stage_mask) {
    if (!b || !stage_mask) return LEE_ERR_ARG;
    *stage_mask = b->band_tile < 0 ? default_band_tile_stages() : b->band_tile;
    return LEE_OK;
}

int lee_batch_fused_tiles(lee_batch *b, long long *fused, long long *total) {
    if (!b || !fused || !total) return LEE_ERR_ARG;
    if (b->dirty) {
        const int rc = batch_refresh(b);
        if (rc != LEE_OK) return rc;
    }
    *fused = b->bv.fuse12 ? b->bv.n_far_tiles : 0;
    *total = b->bv.total_tiles;
    return LEE_OK;
}

int lee_batch_read_latest_probes_async(lee_batch *b, double *host, long long *count) {
    if (!b || !count) return LEE_ERR_ARG;
    if (!b->dev) { b->err = "batch not bound"; return LEE_ERR_ARG; }
    if (b->dirty) {
        const int rc = batch_refresh(b);
        if (rc != LEE_OK) return rc;
    }
    *count = b->nprobe_values;
    if (!host || b->nprobe_values == 0) return LEE_OK;
    cudaError_t e;
    if ((e = launch_probe_latest(b->bv, b->probe_off, b->probe_buf, b->stream)) ||
        (e = cudaMemcpyAsync(host, b->probe_buf, (size_t)b->nprobe_values * 8, cudaMemcpyDeviceToHost, b->stream))) {
        b->err = std::string("batch probes: ") + cudaGetErrorString(e);
        return LEE_ERR_CUDA;
    }
    return LEE_OK;
}

int lee_batch_set_strips_per_sm(lee_batch *b, int strips) {
    if (!b || strips < 0 || strips > 64) return LEE_ERR_ARG;
    b->strips_per_sm = strips ? strips : 2;
    b->dirty = true;
    return LEE_OK;
}

const char *lee_batch_stencil_kernel(lee_batch *b) {
    if (!b || !b->dev) return "";
    if (b->dirty && batch_refresh(b) != LEE_OK) return "";
    return b->members.empty() ? "" : stencil_kernel_name(b->bv);
}

int lee_batch_launch(lee_batch *b, int stage, int what) {
    if (!b || stage < 1 || stage > 4 || what < 0 || what > 1) return LEE_ERR_ARG;
    if (!b->dev) { b->err = "batch not bound"; return LEE_ERR_ARG; }
    if (b->dirty) {
        int rc = batch_refresh(b);
        if (rc != LEE_OK) return rc;
    }
    if (b->members.empty()) return LEE_OK;
    static const int ctas = [] { const char *e = getenv("LEE_STENCIL_CTAS"); return e ? atoi(e) : 0; }();
    cudaError_t e = what == 0 ? launch_ghost(b->bv, stage, b->stream) : launch_stencil(b->bv, stage, ctas, b->stream);
    if (e != cudaSuccess) { b->err = std::string("batch launch: ") + cudaGetErrorString(e); return LEE_ERR_CUDA; }
    return LEE_OK;
}

}  // extern "C"
