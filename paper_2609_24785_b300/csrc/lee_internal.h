// lee_internal.h -- structures shared by the host set-up, the C ABI and the
// CUDA kernels of liblee.  Not part of the public interface (include/lee.h).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

namespace lee {

// Tiles of the fused stencil kernels: TILE_X columns x tile_h rows of outputs.
// FP32 instances without periodic axes use the TMA kernel with 64 x 64 tiles;
// FP64 and periodic instances use the shared-memory kernel with 64 x 32 tiles.
constexpr int TILE_X = 64;
constexpr int TILE_Y = 32;
constexpr int TMA_TILE_Y = 64;
constexpr int GHOST_LANES = 2;          // lanes per ghost point in the ghost kernel
// stencil kernel variants
constexpr int KERNEL_SMEM = 0;          // threads stage the halo box in shared memory (64 x 32 tiles)
constexpr int KERNEL_DIRECT = 1;        // interior tiles read global memory directly (64 x 32 tiles)
constexpr int KERNEL_TMA = 2;           // FP32 TMA pipeline (64 x 64 tiles)
constexpr int GHOST_THREADS = 256;
constexpr int GHOSTS_PER_CTA = GHOST_THREADS / GHOST_LANES;
constexpr int HALO = 4;                 // smem halo on each side (the 7-pt DRP needs 3; 4 keeps
                                        // the TMA box origin 16-byte aligned); band nodes read
                                        // their one-sided windows from global memory
constexpr int MAX_PROBES = 1024;
constexpr int MAX_ADE_STATES = 8;       // ADE states per ghost of a rational admittance (N + 2M)

// status word of an instance (InstDesc::clock[2]), set on the device
constexpr unsigned long long STATUS_TIMEOUT = 1ull;    // a bounded wait for a tile copy gave up
constexpr unsigned long long STATUS_DIVERGED = 2ull;   // a ghost, ADE or probe value is not finite

// tile flags
constexpr uint32_t TILE_BAND = 1u;      // output region meets the 3 outer layers
constexpr uint32_t TILE_MIXED = 2u;     // has non-fluid or out-of-grid outputs
constexpr uint32_t TILE_SPONGE = 4u;    // meets the absorbing ramp along the outer edges
constexpr uint32_t TILE_BAND_FLUID = 8u; // band tile whose band nodes and their 7-node windows are all fluid
constexpr uint32_t TILE_INERT = 32u;    // every node solid, none a ghost: never read by a fluid node's
                                        // stencil, stays zero in every buffer, so no kernel visits it

// Opt-in absorbing ramp along the non-periodic edges (lee_set_sponge; off by
// default, as in the paper): damping rate (kappa / h) ((W - d) / W)^2 at a
// distance d < W cells from the nearest edge.  It removes the slowly growing
// grid-scale modes of the one-sided/radiation closure on long runs.
constexpr int SPONGE_W_DEFAULT = 12;
constexpr double SPONGE_K_DEFAULT = 0.04;

// Per-stage constants of the bulk update of stage k (Sec. 3.2 step 6, Eq. 3):
// alpha_k dt, alpha_k dt a_j / h (j = 1..3), alpha_k dt kappa / h, 1 / h,
// kappa / h (kappa = 0 without the ramp).
enum { K_AD = 0, K_K1 = 1, K_K2 = 2, K_K3 = 3, K_KS = 4, K_INVH = 5, K_SK = 6 };
void fill_stage_constants(double dt, double h, double kappa, float kf[4][8], double kd[4][8]);

// Combined FP64 weight row entry of one cloud node: p_BP = sum l0 p,
// Neumann row wp, Dirichlet row wd, free-extrapolation row wf.
struct alignas(32) GW { double l0, wp, wd, wf; };
// The same 32 bytes for the float-float ghost kernel of the FP32 bulk: each
// FP64 weight w as the pair w = hi + lo of FP32 numbers (hi = fl32(w),
// lo = fl32(w - hi), 48 significant bits), the four hi parts first.
struct alignas(32) GWF { float hi[4], lo[4]; };
static_assert(sizeof(GWF) == sizeof(GW), "both weight layouts take 32 bytes per entry");

// Per-instance descriptor read by every kernel (device copy in the arena;
// copied whole into shared memory in 16-byte pieces by the TMA kernel).
struct alignas(16) InstDesc {
    void *q[3];                 // buffers Q^n, Q^a, Q^b; each holds planes p,u,v
    long long plane;            // elements per plane = ny * pitch
    const uint8_t *mask;        // node kind, ny x pitch (0 solid, 1 fluid, 2 ghost)
    const uint32_t *tile_flags; // tiles_x * tiles_y
    int nx, ny, pitch, tiles_x, tiles_y, ntiles, tile_w, tile_h;
    int per_x, per_y;
    int use_tma;                // FP32 TMA stencil path (kernel_mode == KERNEL_TMA)
    int kernel_mode;            // KERNEL_SMEM / KERNEL_DIRECT / KERNEL_TMA
    const void *tmap[4];        // CUtensorMap (device): halo boxes of Q^n, Q^a, Q^b; 64x64 box of Q^n
    double h, inv_h, dt;
    double cx, cy;              // domain centre in index units ((n-1)/2)
    // ghosts (Sec. 3.1-3.2)
    int ng;
    const int *g_target;        // ng
    const int *g_start;         // ng + 1, entry ranges
    const double2 *g_n;         // ng, wall normal (wall -> fluid)
    const double2 *g_kappa;     // ng, (kappa_p, kappa_u)
    const int *e_idx;           // entries: node index (j * pitch + i)
    const GW *e_w;              // entries: (L0, w_p, w_d, w_f); GWF pairs when
                                // ghost_float_float(precision) holds
    double *Xn;                 // ng x 2 ADE state at t_n
    double *Xs;                 // ng x 2 ADE state of the current stage
    double A[4], b[2], c[2];    // X' = A X + b p_BP, u_n = c . X
    // per-stage constants of the bulk update (index K_*), computed on the host
    // in FP64 so that no kernel does FP64 arithmetic per tile
    float kf[4][8];
    double kd[4][8];
    // monopole source (Sec. 4.3): s = amp * sigma_k * gx[i] * gy[j]
    double s_amp, s_omega;
    double G_re[4], G_im[4];    // stage k: sigma = sin(w t_n) G_re + cos(w t_n) G_im
    const void *gx, *gy;        // source profiles in the bulk precision
    // probes
    int np, pcap;
    const int *p_idx;           // np x 16 node indices (j * pitch + i)
    const double *p_w;          // np x 16 weights
    double *p_hist;             // pcap x np
    long long *clock;           // [0] step in progress, [1] probe records, [2] status
    double *scratch;            // reductions
    double *staging;            // nx * ny doubles for host transfers
    const double *bc;           // ng x 2 boundary data (u.n, dp/dn) of the ghost-fill test hook
    const double *ade;          // ns > 2: A (ns x ns, row-major), b (ns), c (ns) of X' = A X + b p_BP, u_n = c.X
    int ns;                     // ADE states per ghost (2: MSD wall or rigid; N + 2M: rational admittance)
    int precision;
    int sponge_w;               // absorbing ramp width in cells (0: no ramp)
};
static_assert(sizeof(InstDesc) % 16 == 0, "InstDesc is copied in 16-byte pieces");

// Host-side plan of one instance.
struct Plan {
    int nx = 0, ny = 0, pitch = 0;
    int tiles_x = 0, tiles_y = 0, tile_w = TILE_X, tile_h = TILE_Y;
    std::vector<uint8_t> kind;          // ny * nx (host order, no pitch)
    std::vector<uint32_t> tile_flags;
    // ghosts
    std::vector<int> g_target;          // j * nx + i (host order)
    std::vector<int> g_start;
    std::vector<double> g_meta;         // ng x 5: bpx, bpy, nx, ny, r
    std::vector<int> g_m;
    std::vector<double> g_kappa;        // ng x 2
    std::vector<int> e_idx;             // host order j * nx + i
    std::vector<double> e_w;            // 4 per entry
    int n_reduced = 0;
    int n_fluid = 0;
    // ADE
    int regime = 0;
    double A[4] = {0, 0, 0, 0}, b[2] = {0, 0}, c[2] = {0, 0};
    int ns = 2;                         // states per ghost
    std::vector<double> ade_coef;       // ns > 2: A (ns x ns), b (ns), c (ns)
    double ade_amp = 0;
    // probes
    std::vector<int> p_idx;             // np x 16 host order
    std::vector<double> p_w;
};

struct Geometry {
    int kind = 0;               // 0 none, 1 line, 2 cylinder
    double a = 0, b = 0, c = 0; // line: point (a, b), angle c; cylinder: centre (a, b), radius c
};

struct Impedance {
    bool rigid = true;
    double R = 0, M = 0, K = 0;
    // rational admittance (Sec. 2.3, Eq. Yrational with Y_inf = 0): nreal real
    // poles lam with residues A, npair pairs al +- i be with residues B +- i C
    int nreal = 0, npair = 0;
    double lam[MAX_ADE_STATES] = {}, A[MAX_ADE_STATES] = {};
    double al[MAX_ADE_STATES] = {}, be[MAX_ADE_STATES] = {}, B[MAX_ADE_STATES] = {}, C[MAX_ADE_STATES] = {};
    bool rational() const { return !rigid && nreal + npair > 0; }
};

// host set-up (lee_setup.cpp); returns LEE_* status, message in err
int build_plan(int nx, int ny, double h, double x0, double y0, int per_x, int per_y, double dt, int tile_w, int tile_h,
               int sponge_w, const Geometry &geo, const Impedance &imp, const std::vector<double> &probe_xy,
               Plan &plan, std::string &err);
void stage_forcing_factors(double omega, double dt, double G_re[4], double G_im[4]);

// kernel launchers (lee_kernels.cu); all return cudaError_t of the launch
struct BatchView {
    const InstDesc *inst;       // device array of instance descriptors
    int ninst;
    const int *tile_prefix;     // ninst + 1 (device)
    const int4 *ghost_chunks;   // (instance, first ghost, count, 0), one per ghost CTA (device)
    int nchunks;
    const int4 *strips;         // (instance, tile column, first tile row, tiles), longest first (device)
    int nstrips;
    int use_tma;
    int kernel_mode;
    int tile_w, tile_h;
    const int4 *band_chunks;    // band_kernel work list (instance, first band node, count, 0) (device)
    int nband_chunks;           // 0: the stencil kernel does the band itself
    const int *probe_inst;      // instances with probes (device), nprobe_inst entries
    int nprobe_inst;
    int total_tiles;
    int total_ghosts;
    int precision;
    int ade_general;            // some instance has ns > 2: the ghost kernel's general ADE variant
    // fused stages 1 + 2 (lee_batch_set_stage_fusion): tiles clear of walls,
    // band and ramp run pair_kernel; the stencil of stages 1 and 2 takes the
    // other tiles' strips
    int fuse12;
    const int4 *near_strips;    // (instance, tile column, first tile row, tiles) of the other tiles
    int n_near_strips;
    const int4 *far_tiles;      // (instance, x0, y0, 0) of the fused tiles
    int n_far_tiles;
    // stages (bit k for stage k) whose band nodes the warp-specialised stencil
    // does inside its band tiles; band_kernel does them in the other stages
    int band_tile;
};
cudaError_t prepare_kernels(int precision);   // one-time function attributes (outside capture)
int num_sms();
int default_kernel_mode(int precision, bool periodic);
void tma_tile(int &tile_w, int &tile_h);
// TMA descriptors of one FP32 instance (host encode; 4 x 128 bytes)
bool encode_tensor_maps(const InstDesc &d, void *host_out /* 4 x 128 B */, std::string &err);
cudaError_t launch_ghost(const BatchView &bv, int stage, cudaStream_t s);
// FP32 bulk: the ghost projections run in float-float on the FP32 pipe and the
// device weights are stored as GWF (LEE_GHOST_ARITH=f64 selects the FP64 gather)
bool ghost_float_float(int precision);
cudaError_t launch_stencil(const BatchView &bv, int stage, int persistent_ctas, cudaStream_t s);
cudaError_t launch_probes(const BatchView &bv, cudaStream_t s);
// the latest probe record of every instance with probes into dst (instance
// bv.probe_inst[i] at dst + off[i], device arrays)
cudaError_t launch_probe_latest(const BatchView &bv, const int *off, double *dst, cudaStream_t s);
cudaError_t launch_pair(const BatchView &bv, cudaStream_t s);   // fused stages 1 + 2 on bv.far_tiles
int pair_tile_w();
int pair_tile_h();
cudaError_t launch_init(const InstDesc *dinst, const InstDesc &h, int kind, const double *prm, cudaStream_t s);
cudaError_t launch_to_staging(const InstDesc *dinst, const InstDesc &h, int which, int buf, cudaStream_t s);
cudaError_t launch_from_staging(const InstDesc *dinst, const InstDesc &h, int which, cudaStream_t s);
cudaError_t launch_energy(const InstDesc *dinst, const InstDesc &h, cudaStream_t s);
cudaError_t launch_status_gather(const BatchView &bv, long long *out, cudaStream_t s);
const char *stencil_kernel_name(const BatchView &bv);
bool uses_band_pass(int precision, int kernel_mode, int tile_w, int tile_h);
int default_band_tile_stages();         // BatchView::band_tile unless a batch sets its own
bool tma_tile_supported(int tw, int th);
int band_nodes(int nx, int ny, int per_x, int per_y);
// band_kernel work list of one instance (kind: its node kinds, host order)
void band_chunks(int inst, int nband, std::vector<int4> &out, const uint8_t *kind, int nx, int ny);
long long launch_count();
void count_launch(int n = 1);
// message for lee_last_error(NULL) (entry points without a context)
void set_global_error(const std::string &msg);

}  // namespace lee
