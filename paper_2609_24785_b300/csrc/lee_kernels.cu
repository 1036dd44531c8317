// lee_kernels.cu -- CUDA kernels (sm_103a) of one Runge-Kutta stage of the
// ghost-point IBM / ADE / 2D LEE method, for any number of instances per
// launch.
//
//  ghost_kernel       steps 1-5 of Sec. 3.2, GHOST_LANES lanes per ghost point:
//                     gather of the cloud (bulk precision), six projections
//                     with the combined weight rows (FP64 sums; float-float
//                     on the FP32 pipe for the FP32 bulk), the MSD ADE
//                     (Sec. 2.5), the ghost values p, u, v and the ADE update.
//  stencil_ws_kernel  step 6 of Sec. 3.2 (FP32 bulk): 7-point DRP derivatives
//                     (Sec. 2.2 Eq. DRP_s) of the LEE (Sec. 2.1 Eq. 1) from TMA
//                     halo tiles, source, ramp and the 2N-storage stage update
//                     Q(k) = Q(n) + alpha_k dt RHS(Q(k-1)); warp-specialised.
//  band_kernel        the same stage for the fluid nodes of the three outer
//                     layers (one-sided stencils + radiation condition), after
//                     stencil_ws_kernel.
//  stencil_kernel, stencil_tma_kernel
//                     step 6 with the outer band included: shared-memory or
//                     global halo tiles (FP64, periodic axes) and the earlier
//                     3-stage TMA pipeline.
//  probe / init / staging / energy / status kernels: bookkeeping.
#include <atomic>
#include <cstdio>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "lee_internal.h"

namespace lee {

namespace {
std::atomic<long long> g_launches{0};
}
long long launch_count() { return g_launches.load(); }
void count_launch(int n) { g_launches += n; }


// DRP coefficients of Sec. 2.2 (a_{-k} = -a_k)
template <typename T> struct Drp;
template <> struct Drp<float> {
    static constexpr float a1 = 0.770882380518f, a2 = -0.166705904415f, a3 = 0.020843142770f;
};
template <> struct Drp<double> {
    static constexpr double a1 = 0.770882380518, a2 = -0.166705904415, a3 = 0.020843142770;
};

// buffers read / written by stage k (Q^n = 0, Q^a = 1, Q^b = 2)
__host__ __device__ inline int stage_in(int k) { return k == 1 ? 0 : (k == 3 ? 2 : 1); }
__host__ __device__ inline int stage_out(int k) { return k == 4 ? 0 : (k == 2 ? 2 : 1); }

__device__ __forceinline__ int find_inst(const int *__restrict__ prefix, int ninst, int w) {
    int lo = 0, hi = ninst;              // prefix[lo] <= w < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= w) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ GW ldg_gw(const GW *p) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    return GW{a.x, a.y, b.x, b.y};
}

// ---------------------------------------------------------------- ghosts
// FP32 -> FP64 widening on the integer pipe, exact for every input (the
// hardware conversion shares the FP64 pipe with the gather's FMAs): the sign
// moves up, the exponent is rebiased, subnormals are normalised first, the
// mantissa is shifted into place; zeros, infinities and NaNs keep their class.
__device__ __forceinline__ double widen_f32(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned long long bits;
    if (e == 0xffu) {
        bits = 0x7ff0000000000000ull | ((unsigned long long)m << 29);
    } else if (e != 0) {
        bits = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    } else if (m == 0) {
        bits = 0;
    } else {                                        // m 2^-149 = (1 + f) 2^(p - 149)
        const int p = 31 - __clz(m);
        bits = ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
    }
    return __longlong_as_double((long long)(sign | bits));
}
// gather arithmetic of ghost_kernel
enum GhostArith : int {
    GA_F64_HW = 0,              // FP64 sums, hardware FP32 -> FP64 conversion
    GA_F64_INT = 1,             // FP64 sums, integer widening (widen_f32)
    GA_FF = 2                   // float-float sums on the FP32 pipe (FP32 bulk)
};
template <int GA> __device__ __forceinline__ double to_f64(float x) { return GA == GA_F64_INT ? widen_f32(x) : (double)x; }
template <int GA> __device__ __forceinline__ double to_f64(double x) { return x; }

// Float-float dot products (the compensated dot product "Dot2" of Ogita,
// Rump and Oishi, SIAM J. Sci. Comput. 26, 2005), two rows per paired FP32
// instruction.  The weight is the pair w = wh + wl; wh q is split exactly
// into p + e (p = fl(wh q), e = fma(wh, q, -p)), fl(wl q) joins e, p enters
// the running sum through Knuth's exact two-sum and every rounding error is
// collected in the low word.  For n terms the error is about (n 2^-24)^2
// sum|w q| + 2^-48 sum|w q|, against n 2^-53 sum|w q| for FP64 sums: both
// far below the 2^-24 rounding of the stored ghost value.
struct FF2 { float2 hi, lo; };
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void two_sum_acc(FF2 &s, float2 p, float2 e) {
    const float2 t = __fadd2_rn(s.hi, p);
    const float2 bp = __fadd2_rn(t, neg2(s.hi));                 // the part of t that came from p
    const float2 err = __fadd2_rn(__fadd2_rn(s.hi, neg2(__fadd2_rn(t, neg2(bp)))),
                                  __fadd2_rn(p, neg2(bp)));      // s.hi + p - t, exactly
    s.lo = __fadd2_rn(s.lo, __fadd2_rn(err, e));
    s.hi = t;
}
__device__ __forceinline__ void ff_fma(FF2 &s, float2 wh, float2 wl, float2 q) {
    const float2 p = __fmul2_rn(wh, q);
    float2 e = __ffma2_rn(wh, q, neg2(p));                          // wh q - p, exactly
    e = __ffma2_rn(wl, q, e);
    two_sum_acc(s, p, e);
}
__device__ __forceinline__ double ff_value(float hi, float lo) { return (double)hi + (double)lo; }

// Asynchronous global -> shared copies (cp.async, 16 bytes through L2 only,
// 4 bytes through L1): data is fetched early without holding registers.
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One CTA handles GHOSTS_PER_CTA ghosts of one instance (a chunk of the work
// list), GHOST_LANES lanes per ghost point.  stage 1..4: steps 1-5 of Sec. 3.2
// for that stage.  stage 0 (test hook lee_fill_ghosts_with_bc): the ghosts of
// Q^n are filled from the boundary data d.bc (u.n and dp/dn at each boundary
// point) instead of the ADE's, and no ADE state or clock changes.
// GEN: the general ADE of a rational admittance (Sec. 2.3, Eq. ADEgeneral as
// X' = A X + b p_BP, u_n = c . X with d.ns states per ghost and the dense
// coefficients d.ade); GEN = false is the two-state form of the MSD wall
// (Sec. 2.5) and of the rigid wall, with its coefficients in the descriptor.
template <typename T, int GA, bool GEN = false>
__global__ void __launch_bounds__(GHOST_THREADS, GA == GA_FF ? 5 : 0)   // float-float: 5 CTAs per SM; others unconstrained
ghost_kernel(const InstDesc *__restrict__ inst, int ninst, const int4 *__restrict__ chunks, int nchunks,
             int stage) {
    if (stage == 1 && blockIdx.x == 0)
        for (int i = threadIdx.x; i < ninst; i += blockDim.x) inst[i].clock[0] += 1;   // step in progress
    if ((int)blockIdx.x >= nchunks) return;
    const int4 ch = __ldg(chunks + blockIdx.x);
    const int sub = threadIdx.x / GHOST_LANES, lane = threadIdx.x % GHOST_LANES;
    if (sub >= ch.z) return;                        // whole lane groups leave together
    const InstDesc &d = inst[ch.x];
    const int g = ch.y + sub;
    const int e0 = __ldg(d.g_start + g), e1 = __ldg(d.g_start + g + 1);
    // the ADE state of the stage: at stage 1 the step's starting state X^n,
    // which stage 4 of the previous step left in both buffers (so a state
    // upload writes X^n only)
    const double *Xc = stage == 1 ? d.Xn : d.Xs;
    // per-ghost data, fetched before the gather so that the latencies overlap:
    // into registers (FP64 gathers), or by cp.async into shared memory
    // (float-float gather, whose registers go to more resident warps)
    constexpr int NSG = GA == GA_FF ? GHOSTS_PER_CTA : 1;
    __shared__ __align__(16) double2 s_x[NSG], s_xn[NSG], s_n[NSG], s_k[NSG];
    __shared__ int s_t[NSG];
    double x0 = 0, x1 = 0, xn0 = 0, xn1 = 0;
    double2 n = make_double2(0, 0), kap = make_double2(0, 0);
    int t = 0;
    if (lane == 0) {
        if constexpr (GA == GA_FF) {
            if constexpr (!GEN) {
                cp_async16(&s_x[sub], Xc + 2 * g);          // 16-byte aligned: 2 doubles per ghost
                cp_async16(&s_xn[sub], d.Xn + 2 * g);
            }
            cp_async16(&s_n[sub], d.g_n + g);
            cp_async16(&s_k[sub], d.g_kappa + g);
            cp_async4(&s_t[sub], d.g_target + g);
        } else {
            if constexpr (!GEN) {
                x0 = Xc[2 * g]; x1 = Xc[2 * g + 1];
                xn0 = d.Xn[2 * g]; xn1 = d.Xn[2 * g + 1];
            }
            n = __ldg(d.g_n + g);
            kap = __ldg(d.g_kappa + g);
            t = __ldg(d.g_target + g);
        }
    }
    T *P = (T *)d.q[stage == 0 ? 0 : stage_in(stage)];
    T *U = P + d.plane;
    T *V = P + 2 * d.plane;
    const unsigned gmask = ((1u << GHOST_LANES) - 1u) << (threadIdx.x & (32 - GHOST_LANES));
    // rows: s0 = L0 . p -> p_BP (step 1), s1 = w_p . p (Neumann), s2, s3 =
    // w_d . (u, v) (Dirichlet), s4, s5 = w_f . (u, v) (free)
    double s0, s1, s2, s3, s4, s5;
    if constexpr (GA == GA_FF) {
        static_assert(sizeof(T) == 4, "float-float gather is for the FP32 bulk");
        const float4 *W = reinterpret_cast<const float4 *>(d.e_w);
        const float2 z = make_float2(0.f, 0.f);
        FF2 a{z, z}, b{z, z}, c{z, z};                // (s0, s1), (s2, s3), (s4, s5)
        auto accumulate = [&](const float4 &wh, const float4 &wl, float p, float u, float v) {
            ff_fma(a, make_float2(wh.x, wh.y), make_float2(wl.x, wl.y), make_float2(p, p));
            ff_fma(b, make_float2(wh.z, wh.z), make_float2(wl.z, wl.z), make_float2(u, v));
            ff_fma(c, make_float2(wh.w, wh.w), make_float2(wl.w, wl.w), make_float2(u, v));
        };
        // the cloud indices of the next round are loaded one round ahead, so
        // that a round's gathers start without waiting for its index loads
        int e = e0 + lane;
        int ia = e < e1 ? __ldg(d.e_idx + e) : 0;
        int ib = e + GHOST_LANES < e1 ? __ldg(d.e_idx + e + GHOST_LANES) : 0;
        for (; e + GHOST_LANES < e1; e += 2 * GHOST_LANES) {
            const int en = e + 2 * GHOST_LANES;
            const int na = en < e1 ? __ldg(d.e_idx + en) : 0;
            const int nb = en + GHOST_LANES < e1 ? __ldg(d.e_idx + en + GHOST_LANES) : 0;
            const float pa = P[ia], ua = U[ia], va = V[ia];
            const float pb = P[ib], ub = U[ib], vb = V[ib];
            const float4 wha = __ldg(W + 2 * e), wla = __ldg(W + 2 * e + 1);
            const float4 whb = __ldg(W + 2 * (e + GHOST_LANES)), wlb = __ldg(W + 2 * (e + GHOST_LANES) + 1);
            accumulate(wha, wla, pa, ua, va);
            accumulate(whb, wlb, pb, ub, vb);
            ia = na;
            ib = nb;
        }
        if (e < e1) accumulate(__ldg(W + 2 * e), __ldg(W + 2 * e + 1), P[ia], U[ia], V[ia]);
#pragma unroll
        for (int o = GHOST_LANES / 2; o > 0; o >>= 1) {
            auto combine = [&](FF2 &s) {             // add the partner lane's pair
                const float2 oh = make_float2(__shfl_xor_sync(gmask, s.hi.x, o, GHOST_LANES),
                                              __shfl_xor_sync(gmask, s.hi.y, o, GHOST_LANES));
                const float2 ol = make_float2(__shfl_xor_sync(gmask, s.lo.x, o, GHOST_LANES),
                                              __shfl_xor_sync(gmask, s.lo.y, o, GHOST_LANES));
                two_sum_acc(s, oh, ol);
            };
            combine(a);
            combine(b);
            combine(c);
        }
        s0 = ff_value(a.hi.x, a.lo.x); s1 = ff_value(a.hi.y, a.lo.y);
        s2 = ff_value(b.hi.x, b.lo.x); s3 = ff_value(b.hi.y, b.lo.y);
        s4 = ff_value(c.hi.x, c.lo.x); s5 = ff_value(c.hi.y, c.lo.y);
    } else {
        s0 = s1 = s2 = s3 = s4 = s5 = 0;
        auto accumulate = [&](const GW &w, double p, double u, double v) {
            s0 = fma(w.l0, p, s0);
            s1 = fma(w.wp, p, s1);
            s2 = fma(w.wd, u, s2);
            s3 = fma(w.wd, v, s3);
            s4 = fma(w.wf, u, s4);
            s5 = fma(w.wf, v, s5);
        };
        // two entries per lane per round: all loads of both are issued first
        int e = e0 + lane;
        for (; e + GHOST_LANES < e1; e += 2 * GHOST_LANES) {
            const int ia = __ldg(d.e_idx + e), ib = __ldg(d.e_idx + e + GHOST_LANES);
            const GW wa = ldg_gw(d.e_w + e), wb = ldg_gw(d.e_w + e + GHOST_LANES);
            const double pa = to_f64<GA>(P[ia]), ua = to_f64<GA>(U[ia]), va = to_f64<GA>(V[ia]);
            const double pb = to_f64<GA>(P[ib]), ub = to_f64<GA>(U[ib]), vb = to_f64<GA>(V[ib]);
            accumulate(wa, pa, ua, va);
            accumulate(wb, pb, ub, vb);
        }
        if (e < e1) {
            const int ia = __ldg(d.e_idx + e);
            const GW wa = ldg_gw(d.e_w + e);
            accumulate(wa, to_f64<GA>(P[ia]), to_f64<GA>(U[ia]), to_f64<GA>(V[ia]));
        }
#pragma unroll
        for (int o = GHOST_LANES / 2; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(gmask, s0, o, GHOST_LANES);
            s1 += __shfl_xor_sync(gmask, s1, o, GHOST_LANES);
            s2 += __shfl_xor_sync(gmask, s2, o, GHOST_LANES);
            s3 += __shfl_xor_sync(gmask, s3, o, GHOST_LANES);
            s4 += __shfl_xor_sync(gmask, s4, o, GHOST_LANES);
            s5 += __shfl_xor_sync(gmask, s5, o, GHOST_LANES);
        }
    }
    if (lane != 0) return;
    if constexpr (GA == GA_FF) {
        cp_async_wait_all();                           // this thread's own copies
        if constexpr (!GEN) {
            x0 = s_x[sub].x; x1 = s_x[sub].y;
            xn0 = s_xn[sub].x; xn1 = s_xn[sub].y;
        }
        n = s_n[sub];
        kap = s_k[sub];
        t = s_t[sub];
    }
    if (stage == 0) {                                  // test hook: given boundary data
        const double wbp = d.bc[2 * g], dpdn = d.bc[2 * g + 1];
        const double pg = s1 + kap.x * dpdn;
        const double wg = n.x * s2 + n.y * s3 + kap.y * wbp;
        const double tg = -n.y * s4 + n.x * s5;
        P[t] = (T)pg;
        U[t] = (T)(wg * n.x - tg * n.y);
        V[t] = (T)(wg * n.y + tg * n.x);
        return;
    }
    const double pbp = s0;
    if constexpr (GEN) {
        // steps 2-3 for ns states: X' = A X + b p_BP, u_n = c . X, du_n = c . X'
        const int ns = d.ns;
        const double *Am = d.ade, *bv = Am + ns * ns, *cv = bv + ns;
        double xv[MAX_ADE_STATES], xd[MAX_ADE_STATES];
#pragma unroll
        for (int i = 0; i < MAX_ADE_STATES; ++i) xv[i] = i < ns ? Xc[(long long)ns * g + i] : 0.0;
        double un = 0.0, dun = 0.0;
#pragma unroll
        for (int i = 0; i < MAX_ADE_STATES; ++i) {
            if (i < ns) {
                double a = bv[i] * pbp;
#pragma unroll
                for (int j = 0; j < MAX_ADE_STATES; ++j)
                    if (j < ns) a = fma(Am[i * ns + j], xv[j], a);
                xd[i] = a;
                un = fma(cv[i], xv[i], un);
                dun = fma(cv[i], a, dun);
            } else {
                xd[i] = 0.0;
            }
        }
        // steps 4-5 as below
        const double pg = s1 + kap.x * dun;
        const double wg = n.x * s2 + n.y * s3 - kap.y * un;
        const double tg = -n.y * s4 + n.x * s5;
        P[t] = (T)pg;
        U[t] = (T)(wg * n.x - tg * n.y);
        V[t] = (T)(wg * n.y + tg * n.x);
        const double ad = d.kd[stage - 1][K_AD];
        bool fin = isfinite(pbp);
#pragma unroll
        for (int i = 0; i < MAX_ADE_STATES; ++i) {
            if (i < ns) {
                const long long o = (long long)ns * g + i;
                const double y = d.Xn[o] + ad * xd[i];
                d.Xs[o] = y;
                if (stage == 4) d.Xn[o] = y;
                fin = fin && isfinite(y);
            }
        }
        if (!fin) atomicOr((unsigned long long *)&d.clock[2], STATUS_DIVERGED);
        return;
    }
    // step 2: ADE derivative with p_BP as forcing
    const double xd0 = d.A[0] * x0 + d.A[1] * x1 + d.b[0] * pbp;
    const double xd1 = d.A[2] * x0 + d.A[3] * x1 + d.b[1] * pbp;
    // step 3: wall normal velocity (into the wall) and its time derivative
    const double un = d.c[0] * x0 + d.c[1] * x1;
    const double dun = d.c[0] * xd0 + d.c[1] * xd1;
    // steps 4-5: dp/dn = +du_n/dt (Neumann), u.n = -u_n (Dirichlet), free u.tau
    const double pg = s1 + kap.x * dun;
    const double wg = n.x * s2 + n.y * s3 - kap.y * un;
    const double tg = -n.y * s4 + n.x * s5;
    P[t] = (T)pg;
    U[t] = (T)(wg * n.x - tg * n.y);
    V[t] = (T)(wg * n.y + tg * n.x);
    // ADE stage update X(k) = X(n) + alpha_k dt X'
    const double ad = d.kd[stage - 1][K_AD];
    const double y0 = xn0 + ad * xd0, y1 = xn1 + ad * xd1;
    d.Xs[2 * g] = y0;
    d.Xs[2 * g + 1] = y1;
    if (stage == 4) { d.Xn[2 * g] = y0; d.Xn[2 * g + 1] = y1; }
    // divergence: every stage reads the field at the wall, so a non-finite
    // wall pressure or ADE state is flagged within the stage it appears
    if (!(isfinite(pbp) && isfinite(y0) && isfinite(y1)))
        atomicOr((unsigned long long *)&d.clock[2], STATUS_DIVERGED);
}

// ---------------------------------------------------------------- stencil
// Shared-memory halo box: the tile's outputs plus HALO nodes on every side.
constexpr int BOX_X = TILE_X + 2 * HALO;                    // 72
constexpr int THREADS_X = TILE_X / 4;                       // 16 threads across, 4 columns each
constexpr int RY = 4;                                       // rows per thread (shared-memory kernel)

template <typename T> struct alignas(4 * sizeof(T)) Vec4 { T v[4]; };

template <typename T>
__device__ __forceinline__ Vec4<T> ld4(const T *p) { return *reinterpret_cast<const Vec4<T> *>(p); }

template <typename T>
__device__ __forceinline__ T drp(T m3, T m2, T m1, T p1, T p2, T p3) {
    return Drp<T>::a1 * (p1 - m1) + Drp<T>::a2 * (p2 - m2) + Drp<T>::a3 * (p3 - m3);
}

// Derivative rows of the band pass, one per position t of the node in its
// 7-node window along the axis: t = 0, 1, 2 are the one-sided 7-point DRP
// stencils of Tam and Webb (J. Comput. Phys. 107, 1993; the scheme Sec. 2.2
// names for the three outer layers) at nodes 0, 1, 2 from the near edge, t = 3
// the central DRP of Eq. DRP_s, t = 4, 5, 6 the mirror images of rows 2, 1, 0
// at the far edge (row t, column j: -TW[6 - t][6 - j]).
#define LEE_TW0 -2.192280339, 4.748611401, -5.108851915, 4.461567104, -2.833498741, 1.128328861, -0.203876371
#define LEE_TW1 -0.209337622, -1.084875676, 2.147776050, -1.388928322, 0.768949766, -0.281814650, 0.048230454
#define LEE_TW2 0.049041958, -0.468840357, -0.474760914, 1.273274737, -0.518484526, 0.166138533, -0.026369431
#define LEE_BAND_ROWS                                                                                            \
    {{LEE_TW0},                                                                                                  \
     {LEE_TW1},                                                                                                  \
     {LEE_TW2},                                                                                                  \
     {-0.020843142770, 0.166705904415, -0.770882380518, 0.0, 0.770882380518, -0.166705904415, 0.020843142770}, \
     {0.026369431, -0.166138533, 0.518484526, -1.273274737, 0.474760914, 0.468840357, -0.049041958},          \
     {-0.048230454, 0.281814650, -0.768949766, 1.388928322, -2.147776050, 1.084875676, 0.209337622},          \
     {0.203876371, -1.128328861, 2.833498741, -4.461567104, 5.108851915, -4.748611401, 2.192280339}}
__constant__ double c_band_d[7][7] = LEE_BAND_ROWS;
__constant__ float c_band_f[7][7] = LEE_BAND_ROWS;
template <typename T> __device__ __forceinline__ T band_coef(int t, int j);
template <> __device__ __forceinline__ float band_coef<float>(int t, int j) { return c_band_f[t][j]; }
template <> __device__ __forceinline__ double band_coef<double>(int t, int j) { return c_band_d[t][j]; }

// first node of the 7-node window of the derivative at index x of an axis of
// n nodes (n >= 7) and the node's position t in it; periodic axes wrap
__device__ __forceinline__ int band_window(int x, int n, int per, int &t) {
    if (per) { t = 3; return x - 3; }
    const int s = min(max(x - 3, 0), n - 7);
    t = x - s;
    return s;
}

// sum_j C[t][j] (w_j - w_t) / h: the node's own value is taken out of every
// term, which keeps the derivative of a constant exactly zero with rounded
// coefficients
// w[t] by selects (a dynamic index would put the window in local memory)
template <typename T>
__device__ __forceinline__ T pick7(const T (&w)[7], int t) {
    T r = w[0];
#pragma unroll
    for (int j = 1; j < 7; ++j) r = t == j ? w[j] : r;
    return r;
}

template <typename T>
__device__ __forceinline__ T band_deriv(const T (&w)[7], int t, T inv_h) {
    const T wt = pick7(w, t);
    T s = T(0);
#pragma unroll
    for (int j = 0; j < 7; ++j) s += band_coef<T>(t, j) * (w[j] - wt);
    return s * inv_h;
}

// ((W - d) / W)^2 of the opt-in absorbing ramp (width W = d.sponge_w cells,
// 0 = off) at node (gx, gy), 0 outside it (FP32: times the rounded 1 / W
// instead of a division)
template <typename T>
__device__ __forceinline__ T ramp2(const InstDesc &d, int gx, int gy) {
    const int W = d.sponge_w;
    if (W <= 0) return T(0);
    int dist = 1 << 30;
    if (!d.per_x) dist = min(dist, min(gx, d.nx - 1 - gx));
    if (!d.per_y) dist = min(dist, min(gy, d.ny - 1 - gy));
    if (dist >= W) return T(0);
    const T r = sizeof(T) == 4 ? (T)(W - dist) * (T)(1.0f / (float)W) : (T)(W - dist) / (T)W;
    return r * r;
}

// the per-stage constants of an instance in the bulk precision
template <typename T> __device__ __forceinline__ const T *stage_k(const InstDesc &d, int stage);
template <> __device__ __forceinline__ const float *stage_k<float>(const InstDesc &d, int stage) {
    return d.kf[stage - 1];
}
template <> __device__ __forceinline__ const double *stage_k<double>(const InstDesc &d, int stage) {
    return d.kd[stage - 1];
}

__device__ __forceinline__ double stage_sigma(const InstDesc &d, int stage) {
    const double tn = (double)d.clock[0] * d.dt;
    double sn, cs;
    sincos(d.s_omega * tn, &sn, &cs);
    return sn * d.G_re[stage - 1] + cs * d.G_im[stage - 1];
}

// Where Q^n comes from: the halo box itself (stage 1), a shared-memory tile
// box (TMA kernel) or global memory.  (x, y) are tile-local.
template <typename T> struct QnSrc {
    const T *p, *u, *v;
    long long stride;
    __device__ __forceinline__ long long at(int x, int y) const { return (long long)y * stride + x; }
};

// Paired FP32 arithmetic (two lanes per instruction); a - b is the FMA
// b * (-1) + a, which rounds once like a subtraction.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 pair(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// The update of one fluid node (gx, gy) of the three outer layers from its
// 7-node x and y windows of p, u, v (wx, wy; the node is entry tx of wx and
// ty of wy): one-sided DRP stencils (rows 0..2 from an edge) and the radiation
// condition of Tam and Webb dq/dt = -(cos th dq/dx + sin th dq/dy + q / (2 rho)),
// polar about the domain centre, plus the opt-in ramp term; Q^n of the node
// is (qp, qu, qv), the stage values come back in (op, ou, ov).  fx / fy: every
// node of the x / y window is fluid.  Where a wall meets the band, a
// derivative whose window holds a non-fluid node is left out of the radiation
// condition (its one-sided row would feed back ghost values extrapolated from
// clouds clipped by the box).  Every band path calls this, so they agree
// bitwise.
template <typename T>
__device__ __forceinline__ void band_update(const T (&wx)[3][7], const T (&wy)[3][7], int tx, int ty, bool fx,
                                            bool fy, T qp, T qu, T qv, const InstDesc &d, int gx, int gy,
                                            const T *K, T &op, T &ou, T &ov) {
    const T inv_h = K[K_INVH], half_inv_h = T(0.5) * inv_h;
    const T ad = K[K_AD], sk_h = K[K_SK];
    const T dpdx = fx ? band_deriv<T>(wx[0], tx, inv_h) : T(0), dpdy = fy ? band_deriv<T>(wy[0], ty, inv_h) : T(0);
    const T dudx = fx ? band_deriv<T>(wx[1], tx, inv_h) : T(0), dudy = fy ? band_deriv<T>(wy[1], ty, inv_h) : T(0);
    const T dvdx = fx ? band_deriv<T>(wx[2], tx, inv_h) : T(0), dvdy = fy ? band_deriv<T>(wy[2], ty, inv_h) : T(0);
    const T rx = T(gx) - (T)d.cx, ryy = T(gy) - (T)d.cy;
    T ct, st, q2;                                                // cos th, sin th, 1 / (2 h rho)
    if constexpr (sizeof(T) == 4) {
        const float ri = rsqrtf(rx * rx + ryy * ryy);            // FP32: one reciprocal square root
        ct = rx * ri; st = ryy * ri; q2 = half_inv_h * ri;
    } else {
        const T rho = sqrt(rx * rx + ryy * ryy);
        ct = rx / rho; st = ryy / rho; q2 = half_inv_h / rho;
    }
    const T sg = sk_h * ramp2<T>(d, gx, gy);
    const T p0 = pick7(wx[0], tx), u0 = pick7(wx[1], tx), v0 = pick7(wx[2], tx);
    const T rp = -(ct * dpdx + st * dpdy + p0 * q2) - sg * p0;
    const T ru = -(ct * dudx + st * dudy + u0 * q2) - sg * u0;
    const T rv = -(ct * dvdx + st * dvdy + v0 * q2) - sg * v0;
    op = qp + ad * rp;
    ou = qu + ad * ru;
    ov = qv + ad * rv;
}

// band_update() of node (gx, gy) with Q(k-1) read from its global planes gin
// (p; u at +plane; v at +2 plane) and Q^n at (qx, qy) of qn: the windows,
// their mask entries and the three Q^n values are all loaded first, in flight
// together.  Returns false (and no values) for a node that is not fluid.
template <typename T>
__device__ __forceinline__ bool band_values(const T *__restrict__ gin, const QnSrc<T> &qn, int qx, int qy,
                                            const InstDesc &d, int gx, int gy, const T *K, T &op, T &ou, T &ov) {
    const long long plane = d.plane, pitch = d.pitch;
    const long long oq = qn.at(qx, qy);
    const T qp = qn.p[oq], qu = qn.u[oq], qv = qn.v[oq];
    int tx, ty;
    const int sx = band_window(gx, d.nx, d.per_x, tx);
    const int sy = band_window(gy, d.ny, d.per_y, ty);
    T wx[3][7], wy[3][7];
    bool fx = true, fy = true;                   // every node of the window is fluid
    bool self = false;                           // the node itself is fluid
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        int xk = sx + k, yk = sy + k;
        if (d.per_x) xk = (xk % d.nx + d.nx) % d.nx;
        if (d.per_y) yk = (yk % d.ny + d.ny) % d.ny;
        const long long ox = (long long)gy * pitch + xk, oy = (long long)yk * pitch + gx;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            wx[f][k] = gin[f * plane + ox];
            wy[f][k] = gin[f * plane + oy];
        }
        const bool mx = __ldg(d.mask + ox) == 1;
        fx = fx && mx;
        fy = fy && __ldg(d.mask + oy) == 1;
        self = k == tx ? mx : self;
    }
    if (!self) return false;
    band_update<T>(wx, wy, tx, ty, fx, fy, qp, qu, qv, d, gx, gy, K, op, ou, ov);
    return true;
}

// band_values() stored at (gx, gy) of the output planes out.
template <typename T>
__device__ __forceinline__ void band_point(const T *__restrict__ gin, const QnSrc<T> &qn, int qx, int qy,
                                           const InstDesc &d, T *out, int gx, int gy, const T *K) {
    T op, ou, ov;
    if (!band_values<T>(gin, qn, qx, qy, d, gx, gy, K, op, ou, ov)) return;
    const long long o = (long long)gy * d.pitch + gx, plane = d.plane;
    out[o] = op;
    out[plane + o] = ou;
    out[2 * plane + o] = ov;
}

// The band nodes of one tile of the warp-specialised stencil (stages 2-4),
// done by its NC consumer threads (index c) before the tile's regular update,
// from the tile's shared-memory box of Q(k-1) (sp, su, sv: origin at tile
// origin - HALO, BW floats per row) and its shared copy of Q^n (qs: p, u, v
// planes of TW x TH).  Each node's stage values replace its Q^n entries in qs
// (only that node's own update reads them); the regular update then stores
// them with its whole-row vector stores, so no output sector is left half
// written.  Band nodes of the tile, in order: the rows of the top and bottom
// layers across the tile's width, then the left and right layers' columns of
// the other rows; node i goes to warp i % NCW, lane i / NCW (every consumer
// warp takes its share).  TILE_BAND_FLUID tiles (the host found every band
// node and every node of their windows fluid) read the windows from the box;
// a node whose window leaves the box (a last tile 1 or 2 nodes wide or high)
// and every band node of the other tiles read the global planes gin.
template <int TW, int TH, int NC>
__device__ __forceinline__ void band_tile(const float *sp, const float *su, const float *sv, float *qs,
                                          const InstDesc &d, const float *gin, int x0, int y0, uint32_t flags,
                                          const float *K, int c) {
    constexpr int BW = TW + 2 * HALO, BH = TH + 2 * HALO, NCW = NC / 32, QP = TW * TH;
    const int nx = d.nx, ny = d.ny;
    const int w = min(TW, nx - x0), h = min(TH, ny - y0);
    const int ty_lo = max(0, min(3 - y0, h)), ty_hi = max(0, min(y0 + h - (ny - 3), h));
    const int tx_lo = max(0, min(3 - x0, w)), tx_hi = max(0, min(x0 + w - (nx - 3), w));
    const int nrow = (ty_lo + ty_hi) * w, hm = h - ty_lo - ty_hi, cb = tx_lo + tx_hi;
    const int nb = nrow + (hm > 0 ? hm * cb : 0);
    const bool clean = (flags & TILE_BAND_FLUID) != 0;
    const QnSrc<float> qn{qs, qs + QP, qs + 2 * QP, TW};
    for (int i = (c & 31) * NCW + (c >> 5); i < nb; i += NC) {
        int gx, gy;
        if (i < nrow) {
            const int r = i / w, cc = i - r * w;
            gy = r < ty_lo ? y0 + r : y0 + h - ty_hi + (r - ty_lo);
            gx = x0 + cc;
        } else {
            const int j = i - nrow, r = j / cb, cc = j - r * cb;
            gy = y0 + ty_lo + r;
            gx = cc < tx_lo ? x0 + cc : x0 + w - tx_hi + (cc - tx_lo);
        }
        int tx, ty;
        const int bx = band_window(gx, nx, 0, tx) - x0 + HALO;     // box column of the x window
        const int by = band_window(gy, ny, 0, ty) - y0 + HALO;     // box row of the y window
        const int lx = gx - x0, ly = gy - y0, oq = ly * TW + lx;
        float op, ou, ov;
        if (!clean || bx < 0 || bx + 6 >= BW || by < 0 || by + 6 >= BH) {
            if (!band_values<float>(gin, qn, lx, ly, d, gx, gy, K, op, ou, ov)) continue;
        } else {
            float wx[3][7], wy[3][7];
            const int rx = (ly + HALO) * BW + bx, cy = by * BW + lx + HALO;
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                wx[0][k] = sp[rx + k]; wx[1][k] = su[rx + k]; wx[2][k] = sv[rx + k];
                wy[0][k] = sp[cy + k * BW]; wy[1][k] = su[cy + k * BW]; wy[2][k] = sv[cy + k * BW];
            }
            band_update<float>(wx, wy, tx, ty, true, true, qs[oq], qs[QP + oq], qs[2 * QP + oq], d, gx, gy, K,
                               op, ou, ov);
        }
        qs[oq] = op;
        qs[QP + oq] = ou;
        qs[2 * QP + oq] = ov;
    }
}

// Step 6 of Sec. 3.2 on one tile: stage update of every output node owned by
// this thread (4 columns x RY rows).  sp, su, sv point at the box origin
// (tile origin - HALO in x and y) of Q(k-1), bs elements per row: a shared-
// memory halo box, or global memory for interior tiles.  FL is the tile's
// flags, fixed at compile time so that an interior tile (FL == 0) runs the
// DRP update alone:
//   TILE_MIXED: node kinds from the mask; non-fluid nodes get zeros, nodes
//     beyond nx or ny are skipped;
//   TILE_BAND: fluid nodes of the three outer layers are appended to the
//     warp's list (wl_idx, wl_n in shared memory) and then done by the warp's
//     32 lanes together (band_point); no block-wide barrier is involved;
//   TILE_SPONGE: the absorbing-ramp term.
// FP32 (folded form, Eq. 3 with the constants combined):
//   q = q^n - sum_j k_j (f_{+j} - f_{-j}),  k_j = alpha dt a_j / h,
// evaluated two columns per instruction; FP64: q = q^n + alpha dt RHS with
// the DRP derivatives times 1/h.
// QNG: Q^n is in global memory (FP32 then loads it into registers first).
// SKIPBAND: band nodes are not listed; band_kernel does them after this
// kernel, reading Q^n there (stage 4 writes Q(4) over Q^n, so the band nodes
// must keep their Q^n until then), unless BANDST: band_tile() has already put
// their stage values in place of their Q^n entries, and they are stored from
// there with the other nodes.
template <typename T, int RY, int FL, bool QNG, bool SKIPBAND = false, bool BANDST = false>
__device__ __forceinline__ void tile_points(const T *sp, const T *su, const T *sv, const int bs, const QnSrc<T> &qn,
                                            const InstDesc &d, T *out, int xt, int yt, const T *K, T src, int txi,
                                            int tyi, unsigned short *wl_idx, int *wl_n, const T *gin = nullptr) {
    constexpr bool MIXED = (FL & TILE_MIXED) != 0, BAND = (FL & TILE_BAND) != 0, SPONGE = (FL & TILE_SPONGE) != 0;
    constexpr bool FOLD = sizeof(T) == 4;
    const int cx0 = HALO + 4 * txi, ry0 = HALO + RY * tyi;     // box coordinates of the first output
    const int lx0 = 4 * txi, ly0 = RY * tyi;                   // tile-local
    const int gx0 = xt + lx0, gy0 = yt + ly0;
    // only mixed tiles reach past the last column or row; threads there stay
    // for the warp's band pass
    const bool live = !MIXED || (gx0 < d.nx && gy0 < d.ny);
    if (live) {
    const int pitch = d.pitch;
    const long long plane = d.plane;
    const T ad = K[K_AD], inv_h = K[K_INVH];
    const T k1 = K[K_K1], k2 = K[K_K2], k3 = K[K_K3];
    const T ksp = K[K_KS];                        // alpha dt (SPONGE_K / h), folded form
    const T sk_h = K[K_SK];                       // SPONGE_K / h

    // FP32: this thread's Q^n rows are loaded first so that their latency
    // overlaps the shared-memory work below (FP64 loads them row by row to
    // keep its registers)
    constexpr bool PRELOAD = sizeof(T) == 4 && QNG;
    Vec4<T> qn0[PRELOAD ? RY : 1], qn1[PRELOAD ? RY : 1], qn2[PRELOAD ? RY : 1];
    if (PRELOAD) {
#pragma unroll
        for (int r = 0; r < RY; ++r)
            if (!MIXED || gy0 + r < d.ny) {
                qn0[r] = ld4(qn.p + qn.at(lx0, ly0 + r));
                qn1[r] = ld4(qn.u + qn.at(lx0, ly0 + r));
                qn2[r] = ld4(qn.v + qn.at(lx0, ly0 + r));
            }
    }
    // y differences from the thread's 4 columns of p and v (rows -3 .. RY + 2
    // around its outputs), done first so that the column window dies early:
    //   FP32: yv = alpha dt dp/dy, yp = alpha dt dv/dy, two columns per pair;
    //   FP64: dpy = dp/dy, dvy = dv/dy
    float2 yv[FOLD ? RY : 1][2], yp[FOLD ? RY : 1][2];
    T dpy[FOLD ? 1 : RY][4], dvy[FOLD ? 1 : RY][4];
    T vc[SPONGE ? RY : 1][4];                          // v at the outputs (ramp term)
    {
        Vec4<T> cp[RY + 6], cv[RY + 6];
#pragma unroll
        for (int r = 0; r < RY + 6; ++r) {
            cp[r] = ld4(sp + (ry0 - 3 + r) * bs + cx0);
            cv[r] = ld4(sv + (ry0 - 3 + r) * bs + cx0);
        }
#pragma unroll
        for (int r = 0; r < RY; ++r) {
            if constexpr (FOLD) {
                const float2 K1 = dup2(k1), K2 = dup2(k2), K3 = dup2(k3);
#pragma unroll
                for (int P = 0; P < 2; ++P) {
                    auto col = [&](const Vec4<T> &v) { return pair(v.v[2 * P], v.v[2 * P + 1]); };
                    float2 a = __fmul2_rn(K3, sub2(col(cp[r + 6]), col(cp[r])));
                    a = __ffma2_rn(K2, sub2(col(cp[r + 5]), col(cp[r + 1])), a);
                    yv[r][P] = __ffma2_rn(K1, sub2(col(cp[r + 4]), col(cp[r + 2])), a);
                    float2 c = __fmul2_rn(K3, sub2(col(cv[r + 6]), col(cv[r])));
                    c = __ffma2_rn(K2, sub2(col(cv[r + 5]), col(cv[r + 1])), c);
                    yp[r][P] = __ffma2_rn(K1, sub2(col(cv[r + 4]), col(cv[r + 2])), c);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    dpy[r][q] = drp<T>(cp[r].v[q], cp[r + 1].v[q], cp[r + 2].v[q], cp[r + 4].v[q], cp[r + 5].v[q],
                                       cp[r + 6].v[q]) * inv_h;
                    dvy[r][q] = drp<T>(cv[r].v[q], cv[r + 1].v[q], cv[r + 2].v[q], cv[r + 4].v[q], cv[r + 5].v[q],
                                       cv[r + 6].v[q]) * inv_h;
                }
            }
            if (SPONGE) {
#pragma unroll
                for (int q = 0; q < 4; ++q) vc[r][q] = cv[r + 3].v[q];
            }
        }
    }
    T gxv[4] = {T(0), T(0), T(0), T(0)};
    if (src != T(0)) {
        const T *gxs = (const T *)d.gx;
#pragma unroll
        for (int q = 0; q < 4; ++q) gxv[q] = gx0 + q < d.nx ? gxs[gx0 + q] : T(0);
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
        const int gy = gy0 + r;
        if (MIXED && gy >= d.ny) break;
        // node categories: 0 interior fluid, 1 non-fluid (zero), 2 band fluid, 3 outside
        int cat[4] = {0, 0, 0, 0};
        bool simple = true;
        if (MIXED || BAND) {
            uchar4 kind = make_uchar4(1, 1, 1, 1);
            if (MIXED) kind = *reinterpret_cast<const uchar4 *>(d.mask + (long long)gy * pitch + gx0);
            const unsigned char kk[4] = {kind.x, kind.y, kind.z, kind.w};
            const bool yband = BAND && !d.per_y && (gy < 3 || gy > d.ny - 4);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gx = gx0 + q;
                if (MIXED && gx >= d.nx) cat[q] = 3;
                else if (MIXED && kk[q] != 1) cat[q] = 1;
                else if (BAND && (yband || (!d.per_x && (gx < 3 || gx > d.nx - 4)))) cat[q] = 2;
                simple = simple && (cat[q] == 0 || (BANDST && cat[q] == 2));
            }
        }
        T wp[12], wu[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const Vec4<T> a = ld4(sp + (ry0 + r) * bs + cx0 - 4 + 4 * q);
            const Vec4<T> c = ld4(su + (ry0 + r) * bs + cx0 - 4 + 4 * q);
#pragma unroll
            for (int e = 0; e < 4; ++e) { wp[4 * q + e] = a.v[e]; wu[4 * q + e] = c.v[e]; }
        }
        Vec4<T> n0, n1, n2;
        if (PRELOAD) {
            n0 = qn0[r]; n1 = qn1[r]; n2 = qn2[r];
        } else {
            n0 = ld4(qn.p + qn.at(lx0, ly0 + r));
            n1 = ld4(qn.u + qn.at(lx0, ly0 + r));
            n2 = ld4(qn.v + qn.at(lx0, ly0 + r));
        }
        // absorbing ramp ((W - d) / W)^2 of the thread's 4 nodes
        T rr[4] = {T(0), T(0), T(0), T(0)};
        if (SPONGE) {
#pragma unroll
            for (int q = 0; q < 4; ++q) rr[q] = ramp2<T>(d, gx0 + q, gy);
        }
        const T sy = src != T(0) ? src * ((const T *)d.gy)[gy] : T(0);
        Vec4<T> o0, o1, o2;
        if constexpr (FOLD) {
            const float2 K1 = dup2(k1), K2 = dup2(k2), K3 = dup2(k3);
#pragma unroll
            for (int P = 0; P < 2; ++P) {
                const int c = 4 + 2 * P;                       // window index of the pair's first column
                auto col = [&](const Vec4<T> &v) { return pair(v.v[2 * P], v.v[2 * P + 1]); };
                // alpha dt dp/dx
                float2 au = __fmul2_rn(K3, pair(wp[c + 3] - wp[c - 3], wp[c + 4] - wp[c - 2]));
                au = __ffma2_rn(K2, pair(wp[c + 2] - wp[c - 2], wp[c + 3] - wp[c - 1]), au);
                au = __ffma2_rn(K1, pair(wp[c + 1] - wp[c - 1], wp[c + 2] - wp[c]), au);
                // alpha dt (du/dx + dv/dy)
                float2 ap = __ffma2_rn(K3, pair(wu[c + 3] - wu[c - 3], wu[c + 4] - wu[c - 2]), yp[r][P]);
                ap = __ffma2_rn(K2, pair(wu[c + 2] - wu[c - 2], wu[c + 3] - wu[c - 1]), ap);
                ap = __ffma2_rn(K1, pair(wu[c + 1] - wu[c - 1], wu[c + 2] - wu[c]), ap);
                float2 op = sub2(col(n0), ap), ou = sub2(col(n1), au), ov = sub2(col(n2), yv[r][P]);
                if (SPONGE) {
                    const float2 ks = pair(-ksp * rr[2 * P], -ksp * rr[2 * P + 1]);
                    op = __ffma2_rn(ks, pair(wp[c], wp[c + 1]), op);
                    ou = __ffma2_rn(ks, pair(wu[c], wu[c + 1]), ou);
                    ov = __ffma2_rn(ks, pair(vc[r][2 * P], vc[r][2 * P + 1]), ov);
                }
                if (src != T(0)) op = __ffma2_rn(dup2(ad * sy), pair(gxv[2 * P], gxv[2 * P + 1]), op);
                o0.v[2 * P] = op.x; o0.v[2 * P + 1] = op.y;
                o1.v[2 * P] = ou.x; o1.v[2 * P + 1] = ou.y;
                o2.v[2 * P] = ov.x; o2.v[2 * P + 1] = ov.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 + q;
                const T dpdx = drp<T>(wp[c - 3], wp[c - 2], wp[c - 1], wp[c + 1], wp[c + 2], wp[c + 3]) * inv_h;
                const T dudx = drp<T>(wu[c - 3], wu[c - 2], wu[c - 1], wu[c + 1], wu[c + 2], wu[c + 3]) * inv_h;
                T rp = -(dudx + dvy[r][q]);
                if (src != T(0)) rp += sy * gxv[q];
                T ru = -dpdx, rv = -dpy[r][q];
                if (SPONGE && rr[q] != T(0)) {
                    const T sg = sk_h * rr[q];
                    rp -= sg * wp[c]; ru -= sg * wu[c]; rv -= sg * vc[r][q];
                }
                o0.v[q] = n0.v[q] + ad * rp;
                o1.v[q] = n1.v[q] + ad * ru;
                o2.v[q] = n2.v[q] + ad * rv;
            }
        }
        if (BANDST) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (cat[q] == 2) { o0.v[q] = n0.v[q]; o1.v[q] = n1.v[q]; o2.v[q] = n2.v[q]; }
        }
        const long long o = (long long)gy * pitch + gx0;
        if (simple) {
            *reinterpret_cast<Vec4<T> *>(out + o) = o0;
            *reinterpret_cast<Vec4<T> *>(out + plane + o) = o1;
            *reinterpret_cast<Vec4<T> *>(out + 2 * plane + o) = o2;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (cat[q] == 0 || (BANDST && cat[q] == 2)) {
                    out[o + q] = o0.v[q]; out[plane + o + q] = o1.v[q]; out[2 * plane + o + q] = o2.v[q];
                } else if (cat[q] == 1) {
                    out[o + q] = T(0); out[plane + o + q] = T(0); out[2 * plane + o + q] = T(0);
                } else if (cat[q] == 2 && !SKIPBAND) {
                    // at most 4 RY entries per thread, 128 RY per warp
                    wl_idx[atomicAdd(wl_n, 1)] = (unsigned short)(((ly0 + r) << 8) | (lx0 + q));
                }
            }
        }
    }
    }  // live
    if (BAND && !SKIPBAND) {
        __syncwarp();
        const int n = *(volatile int *)wl_n;
        for (int i = threadIdx.x & 31; i < n; i += 32) {
            const int e = wl_idx[i], lx = e & 0xff, ly = e >> 8;
            band_point<T>(gin, qn, lx, ly, d, out, xt + lx, yt + ly, K);
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) *wl_n = 0;
        __syncwarp();
    }
}

// tile_points() with the tile's flags as a compile-time parameter: interior
// tiles get their own code, every other tile the general form (all flags set
// is a superset: each node is classified from the mask, its indices and the
// ramp).  More variants would push the 128-register TMA kernel into spills.
template <typename T, int RY, bool QNG>
__device__ __forceinline__ void tile_dispatch(uint32_t flags, const T *sp, const T *su, const T *sv, const int bs,
                                              const QnSrc<T> &qn, const InstDesc &d, T *out, int xt, int yt,
                                              const T *K, T src, int txi, int tyi, unsigned short *wl_idx,
                                              int *wl_n, const T *gin) {
    if (flags == 0)
        tile_points<T, RY, 0, QNG>(sp, su, sv, bs, qn, d, out, xt, yt, K, src, txi, tyi, wl_idx, wl_n);
    else
        tile_points<T, RY, TILE_BAND | TILE_MIXED | TILE_SPONGE, QNG>(sp, su, sv, bs, qn, d, out, xt, yt, K, src,
                                                                      txi, tyi, wl_idx, wl_n, gin);
}

// Warp-specialised kernel: band nodes are left to band_kernel, which runs
// right after, so band tiles classify their nodes only to skip those; or
// (BANDST) band_tile() has staged their values in the tile's Q^n copy.
template <int RY, bool BANDST>
__device__ __forceinline__ void tile_dispatch_ws(uint32_t flags, const float *sp, const float *su, const float *sv,
                                                 const int bs, const QnSrc<float> &qn, const InstDesc &d, float *out,
                                                 int xt, int yt, const float *K, float src, int txi, int tyi) {
    constexpr int B = TILE_BAND | TILE_SPONGE, M = TILE_BAND | TILE_MIXED | TILE_SPONGE;
    if (flags == 0)
        tile_points<float, RY, 0, false>(sp, su, sv, bs, qn, d, out, xt, yt, K, src, txi, tyi, nullptr, nullptr);
    else if (!(flags & TILE_MIXED))
        tile_points<float, RY, B, false, true, BANDST>(sp, su, sv, bs, qn, d, out, xt, yt, K, src, txi, tyi,
                                                       nullptr, nullptr);
    else
        tile_points<float, RY, M, false, true, BANDST>(sp, su, sv, bs, qn, d, out, xt, yt, K, src, txi, tyi,
                                                       nullptr, nullptr);
}

// per-warp band lists: 128 RY entries per warp, zeroed counters
template <int NWARP, int RY> struct WarpLists {
    unsigned short idx[NWARP][128 * RY];
    int n[NWARP];
    __device__ __forceinline__ void init() {
        for (int w = threadIdx.x; w < NWARP; w += blockDim.x) n[w] = 0;
    }
};

// ---- shared-memory kernel (FP64, periodic instances): 64 x 32 tiles,
// threads load the halo box, Q^n is read from global memory
constexpr int SY = TILE_Y + 2 * HALO;                       // 40 box rows
constexpr int STENCIL_THREADS = THREADS_X * (TILE_Y / RY);  // 128

// DIRECT: interior tiles (all outputs fluid, no band, no ramp) read Q(k-1)
// straight from global memory (neighbour reuse through L1/L2, no barrier);
// the other tiles stage their halo box in shared memory.
template <typename T, bool DIRECT>
__global__ void __launch_bounds__(STENCIL_THREADS)
stencil_kernel(const InstDesc *__restrict__ inst, int ninst, const int *__restrict__ tprefix,
               int total_tiles, int stage) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sp = reinterpret_cast<T *>(smem_raw);
    T *su = sp + SY * BOX_X;
    T *sv = su + SY * BOX_X;
    __shared__ T s_src;
    __shared__ WarpLists<STENCIL_THREADS / 32, RY> wl;
    wl.init();
    __syncthreads();
    const int inb = stage_in(stage), outb = stage_out(stage);
    const int txi = threadIdx.x % THREADS_X, tyi = threadIdx.x / THREADS_X;
    const int wid = threadIdx.x >> 5;

    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int ii = find_inst(tprefix, ninst, tile);
        const InstDesc &d = inst[ii];
        const int lt = tile - __ldg(tprefix + ii);
        const int tx = lt % d.tiles_x, ty = lt / d.tiles_x;
        const int xt = tx * TILE_X, yt = ty * TILE_Y;
        const uint32_t flags = __ldg(d.tile_flags + lt);
        if (flags & TILE_INERT) continue;      // all solid, no ghost: outputs stay zero (whole block)
        const T *qin = (const T *)d.q[inb];
        const long long plane = d.plane;
        const int pitch = d.pitch, nx = d.nx, ny = d.ny;
        T *out = (T *)d.q[outb];
        if (DIRECT && flags == 0) {
            const T *g0 = qin + (long long)(yt - HALO) * pitch + (xt - HALO);
            const T *q0 = (const T *)d.q[0] + (long long)yt * pitch + xt;
            const QnSrc<T> qn{q0, q0 + plane, q0 + 2 * plane, pitch};
            const T src = d.s_amp != 0.0 ? (T)(d.s_amp * stage_sigma(d, stage)) : T(0);
            tile_points<T, RY, 0, true>(g0, g0 + plane, g0 + 2 * plane, pitch, qn, d, out, xt, yt,
                                        stage_k<T>(d, stage), src, txi, tyi, wl.idx[wid], &wl.n[wid]);
            continue;
        }

        // ---- halo box of Q(k-1) into shared memory
        constexpr int C4 = BOX_X / 4;
        for (int e = threadIdx.x; e < SY * C4; e += STENCIL_THREADS) {
            const int r = e / C4, c = (e - r * C4) * 4;
            int gy = yt - HALO + r;
            const int gx = xt - HALO + c;
            Vec4<T> vp, vu, vv;
            if (d.per_x || d.per_y) {
                if (d.per_y) gy = (gy % ny + ny) % ny;
                for (int q = 0; q < 4; ++q) {
                    int x = gx + q;
                    if (d.per_x) x = (x % nx + nx) % nx;
                    const bool in = gy >= 0 && gy < ny && x >= 0 && x < nx;
                    const long long o = (long long)gy * pitch + x;
                    vp.v[q] = in ? qin[o] : T(0);
                    vu.v[q] = in ? qin[plane + o] : T(0);
                    vv.v[q] = in ? qin[2 * plane + o] : T(0);
                }
            } else if (gy >= 0 && gy < ny && gx >= 0 && gx + 3 < pitch) {
                const long long o = (long long)gy * pitch + gx;
                vp = *reinterpret_cast<const Vec4<T> *>(qin + o);
                vu = *reinterpret_cast<const Vec4<T> *>(qin + plane + o);
                vv = *reinterpret_cast<const Vec4<T> *>(qin + 2 * plane + o);
            } else {
                for (int q = 0; q < 4; ++q) vp.v[q] = vu.v[q] = vv.v[q] = T(0);
            }
            *reinterpret_cast<Vec4<T> *>(sp + r * BOX_X + c) = vp;
            *reinterpret_cast<Vec4<T> *>(su + r * BOX_X + c) = vu;
            *reinterpret_cast<Vec4<T> *>(sv + r * BOX_X + c) = vv;
        }
        if (threadIdx.x == 0) s_src = d.s_amp != 0.0 ? (T)(d.s_amp * stage_sigma(d, stage)) : T(0);
        __syncthreads();
        QnSrc<T> qn;
        if (stage == 1) {
            qn = QnSrc<T>{sp + HALO * BOX_X + HALO, su + HALO * BOX_X + HALO, sv + HALO * BOX_X + HALO, BOX_X};
        } else {
            const T *q0 = (const T *)d.q[0] + (long long)yt * pitch + xt;
            qn = QnSrc<T>{q0, q0 + plane, q0 + 2 * plane, pitch};
        }
        tile_dispatch<T, RY, true>(flags, sp, su, sv, BOX_X, qn, d, out, xt, yt, stage_k<T>(d, stage), s_src, txi,
                                   tyi, wl.idx[wid], &wl.n[wid], qin);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- TMA stencil (FP32)
// Persistent CTAs (one per SM) walk vertical strips of 64 x 64 output tiles,
// top to bottom, so that the upper halo rows of a tile were fetched by the
// same SM one tile earlier and are served from L2.  Strips are dealt
// round-robin (longest first).  One thread issues a TMA tensor copy of the
// 72 x 72 halo box of Q(k-1) (p, u, v planes) into one of three shared-memory
// stages, two tiles ahead of the tile being computed; completion is tracked by
// one mbarrier per stage (expect_tx), every wait is bounded.  Q^n is read by
// the threads straight into registers (coalesced 16-byte loads).
// TMA tile geometries: TW x TH outputs, halo box (TW + 8) x (TH + 8) x 3
template <int TW, int TH> struct TmaGeom {
    static constexpr int BW = TW + 2 * HALO, BH = TH + 2 * HALO;
    static constexpr uint32_t BYTES = (uint32_t)BW * BH * 3 * 4;          // one stage
    static constexpr int STAGES = 3;
    static constexpr size_t SMEM = STAGES * (size_t)BYTES + 1024;
    static_assert(BYTES % 128 == 0, "stage size must keep 128-byte alignment");
    static_assert(BW <= 256 && BH <= 256, "TMA box dimensions are at most 256");
};
template <int TW, int TH, int RYT> __host__ __device__ constexpr int tma_threads() { return (TW / 4) * (TH / RYT); }
// CTAs per SM the launch is sized for: two when two CTAs' stages fit in shared
// memory and their threads in the register file at 128 registers each
template <int TW, int TH, int RYT> __host__ __device__ constexpr int tma_ctas_per_sm() {
    return (2 * TmaGeom<TW, TH>::SMEM + 8192 <= 227 * 1024 && tma_threads<TW, TH, RYT>() <= 256) ? 2 : 1;
}
// bounded mbarrier waits: each try_wait may suspend the thread for up to
// WAIT_HINT_NS (it resumes as soon as the phase completes), at most WAIT_SPINS
// times before the wait gives up (milliseconds if the hint is ignored)
constexpr int WAIT_SPINS = 1 << 18;
constexpr uint32_t WAIT_HINT_NS = 20000;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(WAIT_HINT_NS)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < WAIT_SPINS; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// L2 policy for data read once per stage (the Q^n tile of a stage: no other
// tile reads it), so that L2 keeps the halo boxes that neighbouring tiles
// read again (on the sweep: 0.16 GB less DRAM traffic per stage-2 launch)
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tma_load_3d_hint(void *dst, const void *map, uint64_t *bar, int x, int y, int z,
                                                 uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const void *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
            "r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// a bounded wait gave up: flag every instance this block works on
__device__ __noinline__ void flag_block_timeout(const InstDesc *__restrict__ inst, const int4 *__restrict__ strips,
                                                int nstrips) {
    for (int s2 = blockIdx.x; s2 < nstrips; s2 += gridDim.x)
        atomicOr((unsigned long long *)&inst[__ldg(strips + s2).x].clock[2], STATUS_TIMEOUT);
}

template <int TW, int TH, int RYT>
__global__ void __launch_bounds__(tma_threads<TW, TH, RYT>(), (tma_ctas_per_sm<TW, TH, RYT>()))
stencil_tma_kernel(const InstDesc *__restrict__ inst, const int4 *__restrict__ strips, int nstrips, int stage) {
    constexpr int NT = tma_threads<TW, TH, RYT>();
    using G = TmaGeom<TW, TH>;
    constexpr int TMA_STAGES = G::STAGES;
    constexpr uint32_t HALO_BYTES = G::BYTES;
    constexpr int BW = G::BW, BH = G::BH;
    extern __shared__ unsigned char smem_dyn[];
    // 1024-byte aligned start, derived from the shared array so that the
    // compiler keeps shared-memory (not generic) loads
    unsigned char *base = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t bar[TMA_STAGES];
    __shared__ int4 info[TMA_STAGES];  // (instance, x0, y0, flags) of the tile in each stage
    __shared__ float ssrc[TMA_STAGES]; // source amplitude x stage forcing of that tile's instance
    __shared__ WarpLists<NT / 32, RYT> wl;
    __shared__ int s_ntiles;
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    const int inb = stage_in(stage), outb = stage_out(stage);
    // producer cursor (thread 0): strip blockIdx.x + j * gridDim.x, tile row r
    int pj = 0, pr = 0;

    auto issue_next = [&](int b) {            // thread 0: next tile of this CTA into stage b
        const int4 st = __ldg(strips + blockIdx.x + pj * gridDim.x);
        const InstDesc &d = inst[st.x];
        const int ty = st.z + pr;
        const int x0 = st.y * TW, y0 = ty * TH;
        info[b] = make_int4(st.x, x0, y0, (int)__ldg(d.tile_flags + ty * d.tiles_x + st.y));
        ssrc[b] = d.s_amp != 0.0 ? (float)(d.s_amp * stage_sigma(d, stage)) : 0.f;
        mbar_arrive_expect_tx(&bar[b], HALO_BYTES);
        tma_load_3d(base + (size_t)b * HALO_BYTES, d.tmap[inb], &bar[b], x0 - HALO, y0 - HALO, 0);
        if (++pr == st.w) { pr = 0; ++pj; }
    };

    if (tid == 0) {
        int n = 0;
        for (int s = blockIdx.x; s < nstrips; s += gridDim.x) n += __ldg(strips + s).w;
        s_ntiles = n;
        for (int b = 0; b < TMA_STAGES; ++b) mbar_init(&bar[b], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int b = 0; b < TMA_STAGES - 1 && b < n; ++b) issue_next(b);
    }
    wl.init();
    __syncthreads();
    const int ntiles = s_ntiles;
    const int txi = tid % (TW / 4), tyi = tid / (TW / 4);
    for (int k = 0; k < ntiles; ++k) {
        const int b = k % TMA_STAGES;
        const uint32_t parity = (k / TMA_STAGES) & 1;
        // the stage freed at the end of tile k - 1 receives tile k + 2
        if (tid == 0 && k + TMA_STAGES - 1 < ntiles) issue_next((k + TMA_STAGES - 1) % TMA_STAGES);
        if (!mbar_wait_bounded(&bar[b], parity)) atomicExch(&abort_flag, 1);
        const int4 inf = info[b];
        if (!abort_flag) {
            const InstDesc &d = inst[inf.x];
            const float *sp = (const float *)(base + (size_t)b * HALO_BYTES);
            const float *su = sp + BW * BH;
            const float *sv = su + BW * BH;
            QnSrc<float> qn;
            if (stage == 1) {
                qn = QnSrc<float>{sp + HALO * BW + HALO, su + HALO * BW + HALO, sv + HALO * BW + HALO, BW};
            } else {
                const float *q0 = (const float *)d.q[0] + (long long)inf.z * d.pitch + inf.y;
                qn = QnSrc<float>{q0, q0 + d.plane, q0 + 2 * d.plane, d.pitch};
            }
            float *out = (float *)d.q[outb];
            tile_dispatch<float, RYT, true>((uint32_t)inf.w, sp, su, sv, BW, qn, d, out, inf.y, inf.z,
                                            stage_k<float>(d, stage), ssrc[b], txi, tyi, wl.idx[tid >> 5],
                                            &wl.n[tid >> 5], (const float *)d.q[inb]);
        }
        __syncthreads();                               // every thread is done with stage b
        if (abort_flag) {
            // a copy did not complete in time: flag every instance of the block,
            // let each copy issued so far land (tile k's, which timed out, and
            // the ones ahead of it), and leave
            if (tid == 0) {
                flag_block_timeout(inst, strips, nstrips);
                for (int q = 0; q < TMA_STAGES && k + q < ntiles; ++q)
                    mbar_wait_bounded(&bar[(k + q) % TMA_STAGES], ((k + q) / TMA_STAGES) & 1);
            }
            return;
        }
    }
}

// ---------------------------------------------------------------- TMA stencil, warp-specialised (FP32)
// One producer warp and NC / 32 consumer warps per CTA, one CTA per SM.  For
// each tile the producer's lane 0 copies, with TMA tensor loads into one of two
// shared-memory stages, the (TW + 8) x (TH + 8) halo box of Q(k-1) and, from
// stage 2 on, the TW x TH tile of Q^n; a "full" mbarrier per stage counts the
// bytes.  Consumer warps compute the tile from shared memory only and each
// arrives on the stage's "empty" mbarrier when it is done; the producer waits
// for all of them before it refills the stage.  The tile loop has no block-
// wide barrier, so warps drift up to one tile apart and the SM's issue slots
// stay busy across tile boundaries.  Every wait is bounded: one that gives up
// sets STATUS_TIMEOUT on the block's instances, the consumers stop, and the
// producer lets each copy it issued land before the block exits.
template <int TW, int TH, int RYT, int S_> struct WsGeom {
    static constexpr int NC = (TW / 4) * (TH / RYT);           // consumer threads
    static constexpr int NT = NC + 32;                         // + the producer warp
    static constexpr int STAGES = S_;
    static constexpr uint32_t HALO_BYTES = TmaGeom<TW, TH>::BYTES;
    static constexpr uint32_t QN_BYTES = (uint32_t)TW * TH * 3 * 4;
    static constexpr uint32_t STAGE_BYTES = HALO_BYTES + QN_BYTES;
    static constexpr size_t SMEM = STAGES * (size_t)STAGE_BYTES + 1024;
    // static shared memory: band lists, descriptors, barriers
    static constexpr size_t STATIC = STAGES * (sizeof(InstDesc) + 40) + 320;
    // two CTAs per SM when both fit in shared memory and the register file
    static constexpr int CTAS = (2 * (SMEM + STATIC + 1024) <= 228 * 1024 && 2 * NT * 128 <= 65536) ? 2 : 1;
    static_assert(NC % 32 == 0, "whole consumer warps");
    static_assert(HALO_BYTES % 128 == 0 && STAGE_BYTES % 128 == 0, "stage layout keeps 128-byte alignment");
    static_assert(SMEM + STATIC <= 227 * 1024, "the stages must fit in shared memory");
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int TW, int TH, int RYT, int S_, bool BANDT>
__global__ void __launch_bounds__(WsGeom<TW, TH, RYT, S_>::NT, WsGeom<TW, TH, RYT, S_>::CTAS)
stencil_ws_kernel(const InstDesc *__restrict__ inst, const int4 *__restrict__ strips, int nstrips, int stage) {
    using W = WsGeom<TW, TH, RYT, S_>;
    constexpr int S = W::STAGES, NCW = W::NC / 32;
    constexpr int BW = TmaGeom<TW, TH>::BW, BH = TmaGeom<TW, TH>::BH;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *base = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ __align__(8) uint64_t bandbar;     // BANDT: every consumer warp has staged its band nodes
    __shared__ int4 info[S];           // (instance, x0, y0, flags) of the tile in each stage
    __shared__ float ssrc[S];          // source amplitude x stage forcing of that tile's instance
    __shared__ __align__(16) InstDesc sdesc[S];   // the tile's instance descriptor
    __shared__ int s_ntiles;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int inb = stage_in(stage), outb = stage_out(stage);
    if (tid == 0) {
        int n = 0;
        for (int s2 = blockIdx.x; s2 < nstrips; s2 += gridDim.x) n += __ldg(strips + s2).w;
        s_ntiles = n;
        for (int b = 0; b < S; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], NCW);
        }
        mbar_init(&bandbar, NCW);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int ntiles = s_ntiles;

    if (warp == NCW) {
        // ---- producer warp: walks this block's strips (blockIdx.x + j * gridDim.x).
        // Lane 0 waits for the stage and issues the copies; the whole warp
        // copies the tile's instance descriptor into the stage's shared slot,
        // so that consumers read every parameter from shared memory.
        int pj = 0, pr = 0, issued = 0;
        for (int k = 0; k < ntiles; ++k) {
            const int b = k % S;
            // stage b last held tile k - S: wait until every consumer warp is done with it
            int ok = 1;
            if (lane == 0 && k >= S && !mbar_wait_bounded(&empty[b], ((k / S) - 1) & 1)) {
                abort_flag = 1;
                flag_block_timeout(inst, strips, nstrips);
            }
            if (lane == 0) ok = !abort_flag;
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            const int4 st = __ldg(strips + blockIdx.x + pj * gridDim.x);
            const int ty = st.z + pr;
            {
                const int4 *src4 = reinterpret_cast<const int4 *>(inst + st.x);
                int4 *dst4 = reinterpret_cast<int4 *>(&sdesc[b]);
                for (int i = lane; i < (int)(sizeof(InstDesc) / 16); i += 32) dst4[i] = __ldg(src4 + i);
            }
            __syncwarp();
            if (lane == 0) {
                const InstDesc &d = sdesc[b];
                const int x0 = st.y * TW, y0 = ty * TH;
                info[b] = make_int4(st.x, x0, y0, (int)__ldg(d.tile_flags + ty * d.tiles_x + st.y));
                ssrc[b] = d.s_amp != 0.0 ? (float)(d.s_amp * stage_sigma(d, stage)) : 0.f;
                unsigned char *sb = base + (size_t)b * W::STAGE_BYTES;
                mbar_arrive_expect_tx(&full[b], stage == 1 ? W::HALO_BYTES : W::STAGE_BYTES);
                tma_load_3d(sb, d.tmap[inb], &full[b], x0 - HALO, y0 - HALO, 0);
                if (stage != 1)
                    tma_load_3d_hint(sb + W::HALO_BYTES, d.tmap[3], &full[b], x0, y0, 0, policy_evict_first());
            }
            ++issued;
            if (++pr == st.w) { pr = 0; ++pj; }
        }
        if (lane == 0 && abort_flag) {
            // every copy issued must land before the block's shared memory goes away
            for (int j = max(0, issued - S); j < issued; ++j) mbar_wait_bounded(&full[j % S], (j / S) & 1);
        }
        return;
    }

    // ---- consumers
    const int txi = tid % (TW / 4), tyi = tid / (TW / 4);
    int nbandt = 0;                    // band tiles staged so far (BANDT): the parity of bandbar
    for (int k = 0; k < ntiles; ++k) {
        const int b = k % S;
        if (!mbar_wait_bounded(&full[b], (k / S) & 1)) {
            abort_flag = 1;
            if (lane == 0) flag_block_timeout(inst, strips, nstrips);
        }
        if (abort_flag) break;
        const int4 inf = info[b];
        const InstDesc &d = sdesc[b];
        const float *sp = (const float *)(base + (size_t)b * W::STAGE_BYTES);
        const float *su = sp + BW * BH;
        const float *sv = su + BW * BH;
        QnSrc<float> qn;
        if (stage == 1) {
            qn = QnSrc<float>{sp + HALO * BW + HALO, su + HALO * BW + HALO, sv + HALO * BW + HALO, BW};
        } else {
            const float *qs = sp + 3 * BW * BH;
            qn = QnSrc<float>{qs, qs + TW * TH, qs + 2 * TW * TH, TW};
        }
        if (BANDT && (inf.w & TILE_BAND)) {
            // stages 2-4: the band nodes' stage values go into the tile's Q^n
            // copy first; every consumer warp waits until all are in place
            float *qs = reinterpret_cast<float *>(base + (size_t)b * W::STAGE_BYTES) + 3 * BW * BH;
            band_tile<TW, TH, W::NC>(sp, su, sv, qs, d, (const float *)d.q[inb], inf.y, inf.z, (uint32_t)inf.w,
                                     stage_k<float>(d, stage), tid);
            __syncwarp();
            if (lane == 0) mbar_arrive(&bandbar);
            if (!mbar_wait_bounded(&bandbar, nbandt & 1)) {
                abort_flag = 1;
                if (lane == 0) flag_block_timeout(inst, strips, nstrips);
            }
            ++nbandt;
            if (abort_flag) break;
        }
        tile_dispatch_ws<RYT, BANDT>((uint32_t)inf.w, sp, su, sv, BW, qn, d, (float *)d.q[outb], inf.y, inf.z,
                                     stage_k<float>(d, stage), ssrc[b], txi, tyi);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[b]);
    }
}

// ---------------------------------------------------------------- fused stages 1 + 2
// Temporal blocking of the first two stages on tiles clear of walls, of the
// outer band and of the ramp (the host lists them: their region widened by 3
// nodes is fluid and interior, and widened by 8 lies inside the grid; no
// source).  For such a tile T the ghost fill between the stages touches
// nothing the tile reads, so one pass computes
//   Q(1) = Q^n + alpha_1 dt L(Q^n)   on T widened by 4 (in shared memory),
//   Q(2) = Q^n + alpha_2 dt L(Q(1))  on T,
// from one box of Q^n (T widened by 8), and writes Q(1) and Q(2) on T: 9 words
// of traffic per node for the two stages instead of 15.  Both stages run the
// same interior tile code as the stencil kernels (tile_points with no flags),
// so the values are bitwise those of the two separate stages.
constexpr int PAIR_TW = 64, PAIR_TH = 40;                           // the tile shape it serves
constexpr int PAIR_BW = PAIR_TW + 16, PAIR_BH = PAIR_TH + 16;       // Q^n box (halo 8)
constexpr int PAIR_QW = PAIR_TW + 8, PAIR_QH = PAIR_TH + 8;         // Q(1) region (halo 4)
constexpr int PAIR_THREADS = (PAIR_QW / 4) * (PAIR_QH / 2);         // 18 x 24 = 432
constexpr size_t PAIR_SMEM = (size_t)3 * (PAIR_BW * PAIR_BH + PAIR_QW * PAIR_QH) * sizeof(float) + 1024;

__global__ void __launch_bounds__(PAIR_THREADS, 2)
pair_kernel(const InstDesc *__restrict__ inst, const int4 *__restrict__ tiles, int ntiles) {
    extern __shared__ unsigned char smem_dyn[];
    float *box = reinterpret_cast<float *>(smem_dyn + ((16u - (smem_u32(smem_dyn) & 15u)) & 15u));
    float *q1 = box + 3 * PAIR_BW * PAIR_BH;
    __shared__ __align__(16) InstDesc sd;        // the tile's instance, with q1's layout for stage 1
    const int tid = threadIdx.x;
    for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const int4 tl = __ldg(tiles + ti);
        const InstDesc &d = inst[tl.x];
        const int x0 = tl.y, y0 = tl.z;
        {
            const int4 *src4 = reinterpret_cast<const int4 *>(&d);
            int4 *dst4 = reinterpret_cast<int4 *>(&sd);
            for (int i = tid; i < (int)(sizeof(InstDesc) / 16); i += PAIR_THREADS) dst4[i] = src4[i];
        }
        // the Q^n box, 16-byte copies (rows of 80 floats from column x0 - 8)
        const float *qn = (const float *)d.q[0];
        const long long plane = d.plane;
        constexpr int V = PAIR_BW / 4;
        for (int e = tid; e < 3 * PAIR_BH * V; e += PAIR_THREADS) {
            const int f = e / (PAIR_BH * V), r = (e / V) % PAIR_BH, c = (e % V) * 4;
            cp_async16(box + (f * PAIR_BH + r) * PAIR_BW + c,
                       qn + f * plane + (long long)(y0 - 8 + r) * d.pitch + (x0 - 8 + c));
        }
        cp_async_wait_all();
        __syncthreads();
        if (tid == 0) { sd.pitch = PAIR_QW; sd.plane = PAIR_QW * PAIR_QH; }
        __syncthreads();
        // stage 1 on the region widened by 4, into q1 (tile-local coordinates)
        {
            const int txi = tid % (PAIR_QW / 4), tyi = tid / (PAIR_QW / 4);
            const float *sp = box;
            const QnSrc<float> qs{box + 4 * PAIR_BW + 4, box + (PAIR_BH + 4) * PAIR_BW + 4,
                                  box + (2 * PAIR_BH + 4) * PAIR_BW + 4, PAIR_BW};
            tile_points<float, 2, 0, false>(sp, sp + PAIR_BW * PAIR_BH, sp + 2 * PAIR_BW * PAIR_BH, PAIR_BW, qs, sd,
                                            q1, 0, 0, d.kf[0], 0.f, txi, tyi, nullptr, nullptr);
        }
        __syncthreads();
        // Q(1) on the tile to its buffer; stage 2 on the tile
        float *out1 = (float *)d.q[stage_out(1)];
        for (int e = tid; e < 3 * PAIR_TH * (PAIR_TW / 4); e += PAIR_THREADS) {
            const int f = e / (PAIR_TH * (PAIR_TW / 4)), r = (e / (PAIR_TW / 4)) % PAIR_TH, c = (e % (PAIR_TW / 4)) * 4;
            *reinterpret_cast<float4 *>(out1 + f * plane + (long long)(y0 + r) * d.pitch + x0 + c) =
                *reinterpret_cast<const float4 *>(q1 + (f * PAIR_QH + r + 4) * PAIR_QW + 4 + c);
        }
        if (tid < (PAIR_TW / 4) * (PAIR_TH / 2)) {
            const int txi = tid % (PAIR_TW / 4), tyi = tid / (PAIR_TW / 4);
            const QnSrc<float> qs{box + 8 * PAIR_BW + 8, box + (PAIR_BH + 8) * PAIR_BW + 8,
                                  box + (2 * PAIR_BH + 8) * PAIR_BW + 8, PAIR_BW};
            tile_points<float, 2, 0, false>(q1, q1 + PAIR_QW * PAIR_QH, q1 + 2 * PAIR_QW * PAIR_QH, PAIR_QW, qs, d,
                                            (float *)d.q[stage_out(2)], x0, y0, d.kf[1], 0.f, txi, tyi, nullptr,
                                            nullptr);
        }
        __syncthreads();
    }
}

cudaError_t launch_pair(const BatchView &bv, cudaStream_t s) {
    if (bv.n_far_tiles == 0) return cudaSuccess;
    static const cudaError_t attr = cudaFuncSetAttribute(pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)PAIR_SMEM);
    if (attr != cudaSuccess) return attr;
    static const int per_sm = [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_kernel, PAIR_THREADS, PAIR_SMEM) != cudaSuccess ||
            n < 1)
            n = 1;
        return n;
    }();
    const int grid = std::min(bv.n_far_tiles, per_sm * num_sms());
    pair_kernel<<<grid, PAIR_THREADS, PAIR_SMEM, s>>>(bv.inst, bv.far_tiles, bv.n_far_tiles);
    count_launch();
    return cudaGetLastError();
}

int pair_tile_w() { return PAIR_TW; }
int pair_tile_h() { return PAIR_TH; }

// ---------------------------------------------------------------- band pass
// Band node b of a non-periodic instance: rows 0..2 and ny-3..ny-1 over the
// full width (6 nx nodes), then columns 0..2 and nx-3..nx-1 of rows 3..ny-4.
constexpr int BAND_CHUNK = 128;             // band nodes per band_kernel block iteration
// stages whose band nodes the stencil does inside its band tiles by default:
// none (on the 512-instance sweep the in-tile band made the stage-2 launch
// 1.77 ms against 1.43 + 0.20 ms for the stencil and the band pass)
constexpr int BAND_TILE_STAGES = 0;
int band_nodes(int nx, int ny, int per_x, int per_y) {
    return (per_x || per_y || nx < 6 || ny < 6) ? 0 : 6 * nx + 6 * (ny - 6);
}

// band_kernel work list of one instance: chunks of BAND_CHUNK band nodes,
// (instance, first band node, count, 0), one per block iteration
// (chunks whose nodes are all non-fluid, e.g. on the solid side of a straight
// wall, are left out: the kernel would skip each of their nodes)
void band_chunks(int inst, int nband, std::vector<int4> &out, const uint8_t *kind, int nx, int ny) {
    auto node = [&](int b, int &gx, int &gy) {
        if (b < 3 * nx) { gy = b / nx; gx = b % nx; }
        else if (b < 6 * nx) { b -= 3 * nx; gy = ny - 3 + b / nx; gx = b % nx; }
        else { b -= 6 * nx; const int r = b / 6, c = b - 6 * r; gy = 3 + r; gx = c < 3 ? c : nx - 6 + c; }
    };
    for (int f = 0; f < nband; f += BAND_CHUNK) {
        const int cnt = std::min(BAND_CHUNK, nband - f);
        bool any = kind == nullptr;
        for (int b = f; b < f + cnt && !any; ++b) {
            int gx, gy;
            node(b, gx, gy);
            any = kind[(size_t)gy * nx + gx] == 1;
        }
        if (any) out.push_back(make_int4(inst, f, cnt, 0));
    }
}

// After the warp-specialised stencil of a stage: every fluid node of the three
// outer layers is redone by one thread (band_point on the global planes).  A
// block takes whole chunks of one instance, so the instance is known before
// any per-node load; the next chunk's entry is loaded one chunk ahead.  Six
// blocks per SM (80 registers): 7 % faster on the sweep than five at 92 and
// than eight at 64 (spills).
template <typename T>
__global__ void __launch_bounds__(BAND_CHUNK, 6)
band_kernel(const InstDesc *__restrict__ inst, const int4 *__restrict__ chunks, int nchunks, int stage) {
    const int inb = stage_in(stage), outb = stage_out(stage);
    int ci = blockIdx.x;
    int4 ch = ci < nchunks ? __ldg(chunks + ci) : make_int4(0, 0, 0, 0);
    for (; ci < nchunks; ci += gridDim.x) {
        const int cn = ci + gridDim.x;
        const int4 next = cn < nchunks ? __ldg(chunks + cn) : ch;
        if ((int)threadIdx.x < ch.z) {
            const InstDesc &d = inst[ch.x];
            const int nx = d.nx, ny = d.ny;
            int b = ch.y + threadIdx.x, gx, gy;
            if (b < 3 * nx) {
                gy = b / nx; gx = b - gy * nx;
            } else if (b < 6 * nx) {
                b -= 3 * nx; gy = ny - 3 + b / nx; gx = b % nx;
            } else {
                b -= 6 * nx;
                const int r = b / 6, c = b - 6 * r;
                gy = 3 + r; gx = c < 3 ? c : nx - 6 + c;
            }
            const T *P = (const T *)d.q[inb];
            const T *Q0 = (const T *)d.q[0];
            const long long plane = d.plane;
            const QnSrc<T> qn{Q0, Q0 + plane, Q0 + 2 * plane, d.pitch};
            band_point<T>(P, qn, gx, gy, d, (T *)d.q[outb], gx, gy, stage_k<T>(d, stage));
        }
        ch = next;
    }
}

// ---------------------------------------------------------------- probes
template <typename T>
__global__ void probe_kernel(const InstDesc *__restrict__ inst, const int *__restrict__ probe_inst) {
    const InstDesc &d = inst[probe_inst[blockIdx.x]];
    const long long rec = d.clock[1];
    if (rec >= d.pcap) return;
    const T *P = (const T *)d.q[0];
    for (int p = threadIdx.x; p < d.np; p += blockDim.x) {
        double s = 0.0;
        for (int e = 0; e < 16; ++e) s += d.p_w[16 * p + e] * (double)P[d.p_idx[16 * p + e]];
        d.p_hist[rec * d.np + p] = s;
        if (!isfinite(s)) atomicOr((unsigned long long *)&d.clock[2], STATUS_DIVERGED);
    }
    __syncthreads();
    if (threadIdx.x == 0) d.clock[1] = rec + 1;
}

// The latest probe record (record clock[1] - 1) of every instance with probes,
// side by side: instance probe_inst[i]'s values at dst + off[i]; NaN before a
// first record or past the capacity.
__global__ void probe_latest_kernel(const InstDesc *__restrict__ inst, const int *__restrict__ probe_inst,
                                    const int *__restrict__ off, double *__restrict__ dst) {
    const InstDesc &d = inst[probe_inst[blockIdx.x]];
    const long long rec = d.clock[1] - 1;
    double *o = dst + off[blockIdx.x];
    for (int p = threadIdx.x; p < d.np; p += blockDim.x)
        o[p] = rec >= 0 && rec < d.pcap ? d.p_hist[rec * d.np + p] : __longlong_as_double(0x7ff8000000000000LL);
}

cudaError_t launch_probe_latest(const BatchView &bv, const int *off, double *dst, cudaStream_t s) {
    if (bv.nprobe_inst == 0) return cudaSuccess;
    probe_latest_kernel<<<bv.nprobe_inst, 128, 0, s>>>(bv.inst, bv.probe_inst, off, dst);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- init / staging / energy
template <typename T>
__global__ void init_kernel(const InstDesc *__restrict__ dd, int kind, double a0, double a1, double a2,
                            double a3, double a4, double a5, double x0, double y0) {
    const InstDesc &d = *dd;
    const long long n = (long long)d.ny * d.pitch;
    T *P = (T *)d.q[0];
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(o / d.pitch), i = (int)(o - (long long)j * d.pitch);
        double p = 0, u = 0, v = 0;
        if (i < d.nx && d.mask[o] == 1) {
            const double x = x0 + i * d.h, y = y0 + j * d.h;
            if (kind == 0) {               // pulse: a0 = xs, a1 = ys, a2 = amp, a3 = b
                const double dx = x - a0, dy = y - a1;
                p = a2 * exp(-a3 * (dx * dx + dy * dy));
            } else {                       // packet: a0 xs, a1 ys, a2 angle, a3 amp, a4 k, a5 alpha
                const double ca = cos(a2), sa = sin(a2);
                const double s = (x - a0) * ca + (y - a1) * sa;
                p = 0.5 * a3 * exp(-a5 * a5 * s * s) * cos(2.0 * 3.14159265358979323846 * a4 * s);
                u = p * ca;
                v = p * sa;
            }
        }
        P[o] = (T)p;
        P[d.plane + o] = (T)u;
        P[2 * d.plane + o] = (T)v;
    }
}

template <typename T>
__global__ void to_staging_kernel(const InstDesc *__restrict__ dd, int which, int buf) {
    const InstDesc &d = *dd;
    const T *P = (const T *)d.q[buf] + which * d.plane;
    const long long n = (long long)d.nx * d.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(s / d.nx), i = (int)(s - (long long)j * d.nx);
        d.staging[s] = (double)P[(long long)j * d.pitch + i];
    }
}

template <typename T>
__global__ void from_staging_kernel(const InstDesc *__restrict__ dd, int which) {
    const InstDesc &d = *dd;
    T *P = (T *)d.q[0] + which * d.plane;
    const long long n = (long long)d.nx * d.ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(s / d.nx), i = (int)(s - (long long)j * d.nx);
        const long long o = (long long)j * d.pitch + i;
        P[o] = d.mask[o] == 1 ? (T)d.staging[s] : T(0);
    }
}

template <typename T>
__global__ void energy_kernel(const InstDesc *__restrict__ dd) {
    const InstDesc &d = *dd;
    const T *P = (const T *)d.q[0];
    const long long n = (long long)d.ny * d.pitch;
    double acc = 0.0;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        if (d.mask[o] != 1) continue;
        const double p = P[o], u = P[d.plane + o], v = P[2 * d.plane + o];
        acc += p * p + u * u + v * v;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(d.scratch, acc);
}

// status words of a batch's members, in member order
__global__ void status_gather_kernel(const InstDesc *__restrict__ inst, int ninst, long long *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x)
        out[i] = inst[i].clock[2];
}

// ---------------------------------------------------------------- launchers
namespace {
template <typename T> size_t stencil_smem() { return (size_t)3 * SY * BOX_X * sizeof(T); }

template <typename T> cudaError_t setup_stencil_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)stencil_smem<T>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(stencil_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)stencil_smem<T>());
    if (e == cudaSuccess) done = true;
    return e;
}
constexpr int kGridStrideBlocks = 148 * 8;
}  // namespace

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

// stencil kernel of an instance: LEE_FP32_KERNEL / LEE_FP64_KERNEL = tma (FP32
// only), smem or direct; periodic instances use the shared-memory kernels
int default_kernel_mode(int precision, bool periodic) {
    const char *e = getenv(precision == 1 ? "LEE_FP32_KERNEL" : "LEE_FP64_KERNEL");
    const std::string v = e ? e : (precision == 1 ? "tma" : "smem");
    if (v == "direct") return KERNEL_DIRECT;
    if (v == "smem" || periodic || precision != 1) return KERNEL_SMEM;
    return KERNEL_TMA;
}

// warp-specialised TMA kernel (LEE_TMA_WS=0: the 3-stage kernel whose
// threads read Q^n from global memory)
bool tma_ws() {
    static int w = [] {
        const char *e = getenv("LEE_TMA_WS");
        return e ? atoi(e) : 1;
    }();
    return w != 0;
}

// rows per thread of the TMA kernel (4: 256 threads, 2: 512 threads)
int tma_rows() {
    static int r = [] {
        const char *e = getenv("LEE_TMA_RY");
        const int v = e ? atoi(e) : 2;
        return v == 4 ? 4 : 2;
    }();
    return r;
}

template <int TW, int TH, int RYT> cudaError_t tma_attr() {
    return cudaFuncSetAttribute(stencil_tma_kernel<TW, TH, RYT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TmaGeom<TW, TH>::SMEM);
}

template <int TW, int TH, int RYT, int S_> cudaError_t ws_attr() {
    cudaError_t e = cudaFuncSetAttribute(stencil_ws_kernel<TW, TH, RYT, S_, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WsGeom<TW, TH, RYT, S_>::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(stencil_ws_kernel<TW, TH, RYT, S_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)WsGeom<TW, TH, RYT, S_>::SMEM);
}

// stages whose band nodes the warp-specialised stencil does inside its band
// tiles (bit k for stage k) unless a batch chooses; the others leave them to
// band_kernel.  LEE_BAND_TILE overrides (a bit mask, e.g. 0 or 30).
int default_band_tile_stages() {
    static const int m = [] {
        const char *e = getenv("LEE_BAND_TILE");
        return e ? (atoi(e) & 28) : BAND_TILE_STAGES;
    }();
    return m;
}

template <int TW, int TH, int RYT, int S_>
void launch_ws(const BatchView &bv, int stage, int persistent_ctas, cudaStream_t s) {
    using W = WsGeom<TW, TH, RYT, S_>;
    const int grid = std::min(bv.nstrips, persistent_ctas > 0 ? persistent_ctas : W::CTAS * num_sms());
    const int in_tile = grid > 0 && stage >= 2 && ((bv.band_tile >> stage) & 1);
    // grid == 0: no tiles left (every tile fused), only the band pass
    if (grid > 0 && in_tile)
        stencil_ws_kernel<TW, TH, RYT, S_, true><<<grid, W::NT, W::SMEM, s>>>(bv.inst, bv.strips, bv.nstrips, stage);
    else if (grid > 0)
        stencil_ws_kernel<TW, TH, RYT, S_, false><<<grid, W::NT, W::SMEM, s>>>(bv.inst, bv.strips, bv.nstrips, stage);
    if (bv.nband_chunks > 0 && !in_tile) {
        static const int per_sm = [] {
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, band_kernel<float>, BAND_CHUNK, 0) != cudaSuccess || n < 1)
                n = 1;
            return n;
        }();
        const int blocks = std::min(bv.nband_chunks, per_sm * num_sms());
        band_kernel<float><<<blocks, BAND_CHUNK, 0, s>>>(bv.inst, bv.band_chunks, bv.nband_chunks, stage);
        count_launch();
    }
}

// LEE_L2_FETCH=32|64|128: the context's L2 fetch-granularity hint (bytes;
// lasts as long as the process).  Measurement knob; unset leaves the default.
static cudaError_t l2_fetch_hint() {
    static const int bytes = [] {
        const char *e = getenv("LEE_L2_FETCH");
        return e ? atoi(e) : 0;
    }();
    static bool done = false;
    if (done || bytes <= 0) return cudaSuccess;
    done = true;
    return cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes);
}

cudaError_t prepare_kernels(int precision) {
    if (cudaError_t e = l2_fetch_hint(); e != cudaSuccess) return e;
    if (precision == 1) {
        static bool done = false;
        if (!done) {
            cudaError_t e = tma_attr<64, 64, 2>();
            if (e == cudaSuccess) e = tma_attr<64, 64, 4>();
            if (e == cudaSuccess) e = tma_attr<128, 32, 2>();
            if (e == cudaSuccess) e = tma_attr<64, 32, 2>();
            if (e == cudaSuccess) e = ws_attr<64, 60, 2, 2>();
            if (e == cudaSuccess) e = ws_attr<64, 40, 2, 3>();
            if (e == cudaSuccess) e = ws_attr<64, 32, 2, 3>();
            if (e == cudaSuccess) e = ws_attr<64, 24, 2, 2>();
            if (e == cudaSuccess) e = ws_attr<128, 28, 2, 2>();
            if (e != cudaSuccess) return e;
            done = true;
        }
        num_sms();
        return setup_stencil_attr<float>();
    }
    num_sms();
    return setup_stencil_attr<double>();
}

// TMA tile of FP32 instances, LEE_TMA_TILE: warp-specialised kernel 64x40
// (default, three stages), 128x28, 64x60, 64x32 or 64x24; LEE_TMA_WS=0:
// 64x64, 64x32 or 128x32
void tma_tile(int &tw, int &th) {
    static int w = 0, h = 0;
    if (!w) {
        const char *e = getenv("LEE_TMA_TILE");
        const std::string v = e ? e : (tma_ws() ? "64x40" : "64x64");
        if (v == "128x32") { w = 128; h = 32; }
        else if (v == "64x32") { w = 64; h = 32; }
        else if (v == "64x60") { w = 64; h = 60; }
        else if (v == "64x40") { w = 64; h = 40; }
        else if (v == "64x24") { w = 64; h = 24; }
        else if (v == "128x28") { w = 128; h = 28; }
        else { w = 64; h = 64; }
    }
    tw = w; th = h;
}

bool encode_tensor_maps(const InstDesc &d, void *host_out, std::string &err) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            err = "cuTensorMapEncodeTiled is not available";
            return false;
        }
        enc = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    CUtensorMap *maps = (CUtensorMap *)host_out;
    const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, 3};
    const cuuint64_t strides[2] = {(cuuint64_t)d.pitch * 4, (cuuint64_t)d.plane * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t halo_box[3] = {(cuuint32_t)(d.tile_w + 2 * HALO), (cuuint32_t)(d.tile_h + 2 * HALO), 3};
    const cuuint32_t tile_box[3] = {(cuuint32_t)d.tile_w, (cuuint32_t)d.tile_h, 3};   // unused by the kernel
    for (int b = 0; b < 4; ++b) {
        // The halo box rows start 16 bytes before a 256-byte boundary: a 256-byte
        // L2 promotion fetches ~2.7x the row from DRAM, so promotion is off
        // unless LEE_TMA_PROMO asks for it (1: 64 B, 2: 128 B, 3: 256 B).
        static const CUtensorMapL2promotion promo = [] {
            const char *e = getenv("LEE_TMA_PROMO");
            const int v = e ? atoi(e) : 0;
            return v == 1 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
                 : v == 2 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
                 : v == 3 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B : CU_TENSOR_MAP_L2_PROMOTION_NONE;
        }();
        CUresult r = enc(&maps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, d.q[b < 3 ? b : 0], dims, strides,
                         b < 3 ? halo_box : tile_box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         promo, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            err = "cuTensorMapEncodeTiled returned " + std::to_string((int)r);
            return false;
        }
    }
    return true;
}

bool ghost_float_float(int precision) {
    static const bool ff = [] {
        const char *e = getenv("LEE_GHOST_ARITH");
        return !(e && std::string(e) == "f64");
    }();
    return precision == 1 && ff;
}

cudaError_t launch_ghost(const BatchView &bv, int stage, cudaStream_t s) {
    const int blocks = bv.nchunks > 0 ? bv.nchunks : 1;
    static const bool intw = [] {
        const char *e = getenv("LEE_GHOST_WIDEN");
        return !(e && std::string(e) == "hw");
    }();
    const InstDesc *in = bv.inst;
    const int4 *ch = bv.ghost_chunks;
    if (bv.ade_general) {               // some instance has a rational admittance (ns != 2)
        if (ghost_float_float(bv.precision))
            ghost_kernel<float, GA_FF, true><<<blocks, GHOST_THREADS, 0, s>>>(in, bv.ninst, ch, bv.nchunks, stage);
        else if (bv.precision == 1)
            ghost_kernel<float, GA_F64_INT, true><<<blocks, GHOST_THREADS, 0, s>>>(in, bv.ninst, ch, bv.nchunks, stage);
        else
            ghost_kernel<double, GA_F64_HW, true><<<blocks, GHOST_THREADS, 0, s>>>(in, bv.ninst, ch, bv.nchunks, stage);
    } else if (ghost_float_float(bv.precision))
        ghost_kernel<float, GA_FF><<<blocks, GHOST_THREADS, 0, s>>>(in, bv.ninst, ch, bv.nchunks, stage);
    else if (bv.precision == 1 && intw)
        ghost_kernel<float, GA_F64_INT><<<blocks, GHOST_THREADS, 0, s>>>(in, bv.ninst, ch, bv.nchunks, stage);
    else if (bv.precision == 1)
        ghost_kernel<float, GA_F64_HW><<<blocks, GHOST_THREADS, 0, s>>>(in, bv.ninst, ch, bv.nchunks, stage);
    else
        ghost_kernel<double, GA_F64_HW><<<blocks, GHOST_THREADS, 0, s>>>(in, bv.ninst, ch, bv.nchunks, stage);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stencil(const BatchView &bv, int stage, int persistent_ctas, cudaStream_t s) {
    cudaError_t e;
    if (bv.precision == 1 && bv.kernel_mode == KERNEL_TMA) {
        if (bv.total_tiles == 0) return cudaSuccess;
        auto grid_for = [&](int per_sm) {
            return std::min(bv.nstrips, persistent_ctas > 0 ? persistent_ctas : per_sm * num_sms());
        };
        if (bv.tile_w == 64 && bv.tile_h == 32 && !tma_ws()) {
            constexpr int C = tma_ctas_per_sm<64, 32, 2>();
            stencil_tma_kernel<64, 32, 2><<<grid_for(C), tma_threads<64, 32, 2>(), TmaGeom<64, 32>::SMEM, s>>>(
                bv.inst, bv.strips, bv.nstrips, stage);
            count_launch();
            return cudaGetLastError();
        }
        const int grid = grid_for(1);
        if (bv.tile_w == 64 && bv.tile_h == 60)
            launch_ws<64, 60, 2, 2>(bv, stage, persistent_ctas, s);
        else if (bv.tile_w == 64 && bv.tile_h == 40)
            launch_ws<64, 40, 2, 3>(bv, stage, persistent_ctas, s);
        else if (bv.tile_w == 64 && bv.tile_h == 24)
            launch_ws<64, 24, 2, 2>(bv, stage, persistent_ctas, s);
        else if (bv.tile_w == 128 && bv.tile_h == 28)
            launch_ws<128, 28, 2, 2>(bv, stage, persistent_ctas, s);
        else if (bv.tile_w == 64 && bv.tile_h == 32 && tma_ws())
            launch_ws<64, 32, 2, 3>(bv, stage, persistent_ctas, s);
        else if (bv.tile_w == 128)
            stencil_tma_kernel<128, 32, 2><<<grid, tma_threads<128, 32, 2>(), TmaGeom<128, 32>::SMEM, s>>>(
                bv.inst, bv.strips, bv.nstrips, stage);
        else if (tma_rows() == 4)
            stencil_tma_kernel<64, 64, 4><<<grid, tma_threads<64, 64, 4>(), TmaGeom<64, 64>::SMEM, s>>>(
                bv.inst, bv.strips, bv.nstrips, stage);
        else
            stencil_tma_kernel<64, 64, 2><<<grid, tma_threads<64, 64, 2>(), TmaGeom<64, 64>::SMEM, s>>>(
                bv.inst, bv.strips, bv.nstrips, stage);
        count_launch();
        return cudaGetLastError();
    }
    const int grid = persistent_ctas > 0 ? std::min(persistent_ctas, bv.total_tiles) : bv.total_tiles;
    if (bv.kernel_mode == KERNEL_DIRECT) {
        if (bv.precision == 1)
            stencil_kernel<float, true><<<grid, STENCIL_THREADS, stencil_smem<float>(), s>>>(
                bv.inst, bv.ninst, bv.tile_prefix, bv.total_tiles, stage);
        else
            stencil_kernel<double, true><<<grid, STENCIL_THREADS, stencil_smem<double>(), s>>>(
                bv.inst, bv.ninst, bv.tile_prefix, bv.total_tiles, stage);
        count_launch();
        return cudaGetLastError();
    }
    if (bv.precision == 1) {
        if ((e = setup_stencil_attr<float>()) != cudaSuccess) return e;
        stencil_kernel<float, false><<<grid, STENCIL_THREADS, stencil_smem<float>(), s>>>(bv.inst, bv.ninst, bv.tile_prefix,
                                                                                  bv.total_tiles, stage);
    } else {
        if ((e = setup_stencil_attr<double>()) != cudaSuccess) return e;
        stencil_kernel<double, false><<<grid, STENCIL_THREADS, stencil_smem<double>(), s>>>(bv.inst, bv.ninst, bv.tile_prefix,
                                                                                    bv.total_tiles, stage);
    }
    count_launch();
    return cudaGetLastError();
}

// the stencil variant is warp-specialised and leaves the band to band_kernel
bool uses_band_pass(int precision, int kernel_mode, int tile_w, int tile_h) {
    if (precision != 1 || kernel_mode != KERNEL_TMA) return false;
    if (tile_w == 64) return tile_h == 60 || tile_h == 40 || tile_h == 24 || (tile_h == 32 && tma_ws());
    return tile_w == 128 && tile_h == 28;
}

// tile shapes launch_stencil() dispatches for FP32 instances without periodic axes
bool tma_tile_supported(int tw, int th) {
    if (tma_ws())
        return (tw == 128 && th == 28) || (tw == 64 && (th == 60 || th == 40 || th == 32 || th == 24));
    return (tw == 64 && (th == 64 || th == 32)) || (tw == 128 && th == 32);
}

// name of the stencil kernel launch_stencil() picks for a batch view
const char *stencil_kernel_name(const BatchView &bv) {
    if (bv.precision == 1 && bv.kernel_mode == KERNEL_TMA) {
        if (bv.tile_w == 64 && bv.tile_h == 32 && !tma_ws()) return "stencil_tma_kernel<64,32,2>";
        if (bv.tile_w == 64 && bv.tile_h == 60) return "stencil_ws_kernel<64,60,2,2>";
        if (bv.tile_w == 64 && bv.tile_h == 40) return "stencil_ws_kernel<64,40,2,3>";
        if (bv.tile_w == 64 && bv.tile_h == 24) return "stencil_ws_kernel<64,24,2,2>";
        if (bv.tile_w == 64 && bv.tile_h == 32) return "stencil_ws_kernel<64,32,2,3>";
        if (bv.tile_w == 128 && bv.tile_h == 28) return "stencil_ws_kernel<128,28,2,2>";
        if (bv.tile_w == 128) return "stencil_tma_kernel<128,32,2>";
        return tma_rows() == 4 ? "stencil_tma_kernel<64,64,4>" : "stencil_tma_kernel<64,64,2>";
    }
    if (bv.kernel_mode == KERNEL_DIRECT) return bv.precision == 1 ? "stencil_kernel<float,true>" : "stencil_kernel<double,true>";
    return bv.precision == 1 ? "stencil_kernel<float,false>" : "stencil_kernel<double,false>";
}

cudaError_t launch_probes(const BatchView &bv, cudaStream_t s) {
    if (bv.nprobe_inst == 0) return cudaSuccess;
    if (bv.precision == 1) probe_kernel<float><<<bv.nprobe_inst, 256, 0, s>>>(bv.inst, bv.probe_inst);
    else probe_kernel<double><<<bv.nprobe_inst, 256, 0, s>>>(bv.inst, bv.probe_inst);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_init(const InstDesc *dinst, const InstDesc &h, int kind, const double *prm, cudaStream_t s) {
    const long long n = (long long)h.ny * h.pitch;
    const int blocks = (int)std::min<long long>((n + 255) / 256, kGridStrideBlocks);
    if (h.precision == 1)
        init_kernel<float><<<blocks, 256, 0, s>>>(dinst, kind, prm[0], prm[1], prm[2], prm[3], prm[4], prm[5], prm[6], prm[7]);
    else
        init_kernel<double><<<blocks, 256, 0, s>>>(dinst, kind, prm[0], prm[1], prm[2], prm[3], prm[4], prm[5], prm[6], prm[7]);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_to_staging(const InstDesc *dinst, const InstDesc &h, int which, int buf, cudaStream_t s) {
    const long long n = (long long)h.nx * h.ny;
    const int blocks = (int)std::min<long long>((n + 255) / 256, kGridStrideBlocks);
    if (h.precision == 1) to_staging_kernel<float><<<blocks, 256, 0, s>>>(dinst, which, buf);
    else to_staging_kernel<double><<<blocks, 256, 0, s>>>(dinst, which, buf);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_from_staging(const InstDesc *dinst, const InstDesc &h, int which, cudaStream_t s) {
    const long long n = (long long)h.nx * h.ny;
    const int blocks = (int)std::min<long long>((n + 255) / 256, kGridStrideBlocks);
    if (h.precision == 1) from_staging_kernel<float><<<blocks, 256, 0, s>>>(dinst, which);
    else from_staging_kernel<double><<<blocks, 256, 0, s>>>(dinst, which);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_energy(const InstDesc *dinst, const InstDesc &h, cudaStream_t s) {
    const long long n = (long long)h.ny * h.pitch;
    const int blocks = (int)std::min<long long>((n + 255) / 256, kGridStrideBlocks);
    if (h.precision == 1) energy_kernel<float><<<blocks, 256, 0, s>>>(dinst);
    else energy_kernel<double><<<blocks, 256, 0, s>>>(dinst);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_status_gather(const BatchView &bv, long long *out, cudaStream_t s) {
    if (bv.ninst <= 0) return cudaSuccess;
    status_gather_kernel<<<(bv.ninst + 255) / 256, 256, 0, s>>>(bv.inst, bv.ninst, out);
    count_launch();
    return cudaGetLastError();
}

}  // namespace lee
