// lee_kernels.cu -- CUDA kernels (sm_103a) of one Runge-Kutta stage of the
// ghost-point IBM / ADE / 2D LEE method, for any number of instances per
// launch.
//
//  ghost_kernel    steps 1-5 of Sec. 3.2, one warp per ghost point: gather of
//                  the cloud (bulk precision), six FP64 projections with the
//                  combined weight rows, the MSD ADE (Sec. 2.5), the ghost
//                  values p, u, v and the ADE stage update.
//  stencil_kernel  step 6 of Sec. 3.2: 7-point DRP derivatives (Sec. 2.2 Eq.
//                  DRP_s) of the LEE (Sec. 2.1 Eq. 1) from a shared-memory halo
//                  tile, one-sided stencils + radiation condition in the outer
//                  band, source, and the 2N-storage stage update
//                  Q(k) = Q(n) + alpha_k dt RHS(Q(k-1)).
//  probe / init / staging / energy kernels: bookkeeping.
#include <atomic>
#include <cstdio>
#include <string>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "lee_internal.h"

namespace lee {

namespace {
std::atomic<long long> g_launches{0};
}
long long launch_count() { return g_launches.load(); }
void count_launch(int n) { g_launches += n; }

__constant__ double c_alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};

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
// One CTA handles GHOSTS_PER_CTA ghosts of one instance (a chunk of the work
// list), GHOST_LANES lanes per ghost point.
template <typename T>
__global__ void __launch_bounds__(GHOST_THREADS)
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
    // per-ghost data, fetched before the gather so that the latencies overlap
    double x0 = 0, x1 = 0, xn0 = 0, xn1 = 0;
    double2 n = make_double2(0, 0), kap = make_double2(0, 0);
    int t = 0;
    if (lane == 0) {
        x0 = d.Xs[2 * g]; x1 = d.Xs[2 * g + 1];
        xn0 = d.Xn[2 * g]; xn1 = d.Xn[2 * g + 1];
        n = __ldg(d.g_n + g);
        kap = __ldg(d.g_kappa + g);
        t = __ldg(d.g_target + g);
    }
    T *P = (T *)d.q[stage_in(stage)];
    T *U = P + d.plane;
    T *V = P + 2 * d.plane;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
    for (int e = e0 + lane; e < e1; e += GHOST_LANES) {
        const int idx = __ldg(d.e_idx + e);
        const GW w = ldg_gw(d.e_w + e);
        const double p = (double)P[idx], u = (double)U[idx], v = (double)V[idx];
        s0 = fma(w.l0, p, s0);       // L0 . p      -> p_BP          (step 1)
        s1 = fma(w.wp, p, s1);       // w_p . p     (Neumann row)
        s2 = fma(w.wd, u, s2);       // w_d . u     (Dirichlet row)
        s3 = fma(w.wd, v, s3);
        s4 = fma(w.wf, u, s4);       // w_f . u     (free row)
        s5 = fma(w.wf, v, s5);
    }
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
#pragma unroll
    for (int o = GHOST_LANES / 2; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(gmask, s0, o, GHOST_LANES);
        s1 += __shfl_xor_sync(gmask, s1, o, GHOST_LANES);
        s2 += __shfl_xor_sync(gmask, s2, o, GHOST_LANES);
        s3 += __shfl_xor_sync(gmask, s3, o, GHOST_LANES);
        s4 += __shfl_xor_sync(gmask, s4, o, GHOST_LANES);
        s5 += __shfl_xor_sync(gmask, s5, o, GHOST_LANES);
    }
    if (lane != 0) return;
    const double pbp = s0;
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
    const double ad = c_alpha[stage - 1] * d.dt;
    const double y0 = xn0 + ad * xd0, y1 = xn1 + ad * xd1;
    d.Xs[2 * g] = y0;
    d.Xs[2 * g + 1] = y1;
    if (stage == 4) { d.Xn[2 * g] = y0; d.Xn[2 * g + 1] = y1; }
}

// ---------------------------------------------------------------- stencil
constexpr int SX = TILE_X + 2 * HALO;   // 72 smem columns
constexpr int SY = TILE_Y + 2 * HALO;   // 40 smem rows
constexpr int THREADS_X = TILE_X / 4;   // 16 threads across, 4 columns each
constexpr int THREADS_Y = 8;
constexpr int RY = TILE_Y / THREADS_Y;  // 4 rows per thread
constexpr int STENCIL_THREADS = THREADS_X * THREADS_Y;

template <typename T> struct alignas(4 * sizeof(T)) Vec4 { T v[4]; };

template <typename T>
__device__ __forceinline__ Vec4<T> lds4(const T *p) { return *reinterpret_cast<const Vec4<T> *>(p); }

template <typename T>
__device__ __forceinline__ T drp(T m3, T m2, T m1, T p1, T p2, T p3) {
    return Drp<T>::a1 * (p1 - m1) + Drp<T>::a2 * (p2 - m2) + Drp<T>::a3 * (p3 - m3);
}

// derivative along one axis at absolute index x (axis length n) from smem
// values f(k) = value at absolute index x + k; one-sided rows in the band
template <typename T, typename F>
__device__ __forceinline__ T deriv_general(F f, int x, int n, int per, T inv_h) {
    if (per || (x >= 3 && x <= n - 4)) return drp<T>(f(-3), f(-2), f(-1), f(1), f(2), f(3)) * inv_h;
    const T i12 = inv_h / T(12);
    if (x == 0) return (T(-25) * f(0) + T(48) * f(1) - T(36) * f(2) + T(16) * f(3) - T(3) * f(4)) * i12;
    if (x == 1) return (T(-3) * f(-1) - T(10) * f(0) + T(18) * f(1) - T(6) * f(2) + f(3)) * i12;
    if (x == 2) return (f(-2) - T(8) * f(-1) + T(8) * f(1) - f(2)) * i12;
    if (x == n - 1) return (T(25) * f(0) - T(48) * f(-1) + T(36) * f(-2) - T(16) * f(-3) + T(3) * f(-4)) * i12;
    if (x == n - 2) return (T(3) * f(1) + T(10) * f(0) - T(18) * f(-1) + T(6) * f(-2) - f(-3)) * i12;
    return (f(-2) - T(8) * f(-1) + T(8) * f(1) - f(2)) * i12;              // x == n - 3
}

template <typename T>
__device__ __forceinline__ double stage_sigma(const InstDesc &d, int stage) {
    const double tn = (double)d.clock[0] * d.dt;
    double sn, cs;
    sincos(d.s_omega * tn, &sn, &cs);
    return sn * d.G_re[stage - 1] + cs * d.G_im[stage - 1];
}

template <typename T>
__global__ void __launch_bounds__(STENCIL_THREADS)
stencil_kernel(const InstDesc *__restrict__ inst, int ninst, const int *__restrict__ tprefix,
               int total_tiles, int stage) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T (*sp)[SX] = reinterpret_cast<T (*)[SX]>(smem_raw);
    T (*su)[SX] = sp + SY;
    T (*sv)[SX] = su + SY;
    __shared__ T s_src;
    const int inb = stage_in(stage), outb = stage_out(stage);
    const int txi = threadIdx.x % THREADS_X, tyi = threadIdx.x / THREADS_X;

    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int ii = find_inst(tprefix, ninst, tile);
        const InstDesc &d = inst[ii];
        const int lt = tile - __ldg(tprefix + ii);
        const int tx = lt % d.tiles_x, ty = lt / d.tiles_x;
        const int xt = tx * TILE_X, yt = ty * TILE_Y;
        const uint32_t flags = __ldg(d.tile_flags + lt);
        const T *qin = (const T *)d.q[inb];
        const long long plane = d.plane;
        const int pitch = d.pitch, nx = d.nx, ny = d.ny;

        // ---- halo tile of Q(k-1) into shared memory
        constexpr int C4 = SX / 4;
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
            *reinterpret_cast<Vec4<T> *>(&sp[r][c]) = vp;
            *reinterpret_cast<Vec4<T> *>(&su[r][c]) = vu;
            *reinterpret_cast<Vec4<T> *>(&sv[r][c]) = vv;
        }
        if (threadIdx.x == 0) s_src = d.s_amp != 0.0 ? (T)(d.s_amp * stage_sigma<T>(d, stage)) : T(0);
        __syncthreads();

        const T inv_h = (T)d.inv_h;
        const T ad = (T)(c_alpha[stage - 1] * d.dt);
        const T src = s_src;
        const T *gxs = (const T *)d.gx;
        const T *gys = (const T *)d.gy;
        T *out = (T *)d.q[outb];
        const T *qn = (const T *)d.q[0];
        const int cx0 = HALO + 4 * txi;          // smem column of this thread's first output
        const int ry0 = HALO + RY * tyi;         // smem row of this thread's first output
        const int gx0 = xt + 4 * txi;
        const int gy0 = yt + RY * tyi;

        if (flags == 0) {
            // ---- interior fast path: all outputs fluid, no band
            T dpdy[RY][4], dvdy[RY][4];
            {
                T cp[RY + 6][4], cv[RY + 6][4];
#pragma unroll
                for (int r = 0; r < RY + 6; ++r) {
                    const Vec4<T> a = lds4(&sp[ry0 - 3 + r][cx0]);
                    const Vec4<T> b = lds4(&sv[ry0 - 3 + r][cx0]);
#pragma unroll
                    for (int c = 0; c < 4; ++c) { cp[r][c] = a.v[c]; cv[r][c] = b.v[c]; }
                }
#pragma unroll
                for (int r = 0; r < RY; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        dpdy[r][c] = drp<T>(cp[r][c], cp[r + 1][c], cp[r + 2][c], cp[r + 4][c], cp[r + 5][c], cp[r + 6][c]);
                        dvdy[r][c] = drp<T>(cv[r][c], cv[r + 1][c], cv[r + 2][c], cv[r + 4][c], cv[r + 5][c], cv[r + 6][c]);
                    }
            }
#pragma unroll
            for (int r = 0; r < RY; ++r) {
                T wp[12], wu[12];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const Vec4<T> a = lds4(&sp[ry0 + r][cx0 - 4 + 4 * q]);
                    const Vec4<T> b = lds4(&su[ry0 + r][cx0 - 4 + 4 * q]);
#pragma unroll
                    for (int c = 0; c < 4; ++c) { wp[4 * q + c] = a.v[c]; wu[4 * q + c] = b.v[c]; }
                }
                const int gy = gy0 + r;
                const long long o = (long long)gy * pitch + gx0;
                Vec4<T> n0, n1, n2;
                if (stage == 1) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) { n0.v[c] = wp[4 + c]; n1.v[c] = wu[4 + c]; n2.v[c] = sv[ry0 + r][cx0 + c]; }
                } else {
                    n0 = *reinterpret_cast<const Vec4<T> *>(qn + o);
                    n1 = *reinterpret_cast<const Vec4<T> *>(qn + plane + o);
                    n2 = *reinterpret_cast<const Vec4<T> *>(qn + 2 * plane + o);
                }
                Vec4<T> o0, o1, o2;
                const T gyv = src != T(0) ? gys[gy] : T(0);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = 4 + c;
                    const T dpdx = drp<T>(wp[k - 3], wp[k - 2], wp[k - 1], wp[k + 1], wp[k + 2], wp[k + 3]) * inv_h;
                    const T dudx = drp<T>(wu[k - 3], wu[k - 2], wu[k - 1], wu[k + 1], wu[k + 2], wu[k + 3]) * inv_h;
                    T rp = -(dudx + dvdy[r][c] * inv_h);
                    if (src != T(0)) rp += src * gxs[gx0 + c] * gyv;
                    o0.v[c] = n0.v[c] + ad * rp;
                    o1.v[c] = n1.v[c] - ad * dpdx;
                    o2.v[c] = n2.v[c] - ad * (dpdy[r][c] * inv_h);
                }
                *reinterpret_cast<Vec4<T> *>(out + o) = o0;
                *reinterpret_cast<Vec4<T> *>(out + plane + o) = o1;
                *reinterpret_cast<Vec4<T> *>(out + 2 * plane + o) = o2;
            }
        } else {
            // ---- general path: band (one-sided + radiation), mask, ragged edges
            const T half_inv_h = T(0.5) * inv_h;
            for (int r = 0; r < RY; ++r) {
                const int gy = gy0 + r, sr = ry0 + r;
                if (gy >= ny) break;
                for (int c = 0; c < 4; ++c) {
                    const int gx = gx0 + c, sc = cx0 + c;
                    if (gx >= nx) break;
                    const long long o = (long long)gy * pitch + gx;
                    const uint8_t kind = (flags & TILE_MIXED) ? __ldg(d.mask + o) : (uint8_t)1;
                    if (kind != 1) {
                        out[o] = T(0); out[plane + o] = T(0); out[2 * plane + o] = T(0);
                        continue;
                    }
                    const bool band = (!d.per_x && (gx < 3 || gx > nx - 4)) || (!d.per_y && (gy < 3 || gy > ny - 4));
                    auto fxp = [&](int k) { return sp[sr][sc + k]; };
                    auto fxu = [&](int k) { return su[sr][sc + k]; };
                    auto fyp = [&](int k) { return sp[sr + k][sc]; };
                    auto fyv = [&](int k) { return sv[sr + k][sc]; };
                    const T dpdx = deriv_general<T>(fxp, gx, nx, d.per_x, inv_h);
                    const T dpdy = deriv_general<T>(fyp, gy, ny, d.per_y, inv_h);
                    T rp, ru, rv;
                    if (!band) {
                        const T dudx = deriv_general<T>(fxu, gx, nx, d.per_x, inv_h);
                        const T dvdy = deriv_general<T>(fyv, gy, ny, d.per_y, inv_h);
                        rp = -(dudx + dvdy);
                        if (src != T(0)) rp += src * gxs[gx] * gys[gy];
                        ru = -dpdx;
                        rv = -dpdy;
                    } else {
                        auto fyu = [&](int k) { return su[sr + k][sc]; };
                        auto fxv = [&](int k) { return sv[sr][sc + k]; };
                        const T dudx = deriv_general<T>(fxu, gx, nx, d.per_x, inv_h);
                        const T dudy = deriv_general<T>(fyu, gy, ny, d.per_y, inv_h);
                        const T dvdx = deriv_general<T>(fxv, gx, nx, d.per_x, inv_h);
                        const T dvdy = deriv_general<T>(fyv, gy, ny, d.per_y, inv_h);
                        const T rx = T(gx) - (T)d.cx, ryy = T(gy) - (T)d.cy;
                        const T rho = sqrt(rx * rx + ryy * ryy);
                        const T ct = rx / rho, st = ryy / rho;
                        const T q2 = half_inv_h / rho;      // 1 / (2 h rho)
                        rp = -(ct * dpdx + st * dpdy + sp[sr][sc] * q2);
                        ru = -(ct * dudx + st * dudy + su[sr][sc] * q2);
                        rv = -(ct * dvdx + st * dvdy + sv[sr][sc] * q2);
                    }
                    const T n0 = stage == 1 ? sp[sr][sc] : qn[o];
                    const T n1 = stage == 1 ? su[sr][sc] : qn[plane + o];
                    const T n2 = stage == 1 ? sv[sr][sc] : qn[2 * plane + o];
                    out[o] = n0 + ad * rp;
                    out[plane + o] = n1 + ad * ru;
                    out[2 * plane + o] = n2 + ad * rv;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- TMA stencil (FP32)
// Persistent CTAs (one per SM) walk the tile list.  For every 64 x 64 output
// tile one thread issues two TMA tensor copies into a shared-memory stage: the
// 72 x 72 halo box of Q(k-1) (p, u, v planes) and, for stages 2-4, the 64 x 64
// box of Q^n.  Two stages are in flight: while tile i is computed from one
// stage, the copies of tile i + 1 land in the other.  Completion is tracked by
// one mbarrier per stage (expect_tx); every wait is bounded.
constexpr int TB_X = TILE_X + 2 * HALO;                     // 72
constexpr int TB_Y = TMA_TILE_Y + 2 * HALO;                 // 72
constexpr int TMA_THREADS = 256;
constexpr int TMA_TX = TILE_X / 4;                          // 16 threads across, 4 columns each
constexpr int TMA_TY = TMA_THREADS / TMA_TX;                // 16 threads down
constexpr int TMA_RY = TMA_TILE_Y / TMA_TY;                 // 4 rows each
constexpr uint32_t HALO_BYTES = TB_X * TB_Y * 3 * 4;        // 62208
constexpr uint32_t QN_BYTES = TILE_X * TMA_TILE_Y * 3 * 4;  // 49152
constexpr uint32_t STAGE_BYTES = HALO_BYTES + QN_BYTES;     // 111360 = 870 x 128
constexpr size_t TMA_SMEM = 2 * (size_t)STAGE_BYTES + 1024;
constexpr int WAIT_SPINS = 1 << 20;

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
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < WAIT_SPINS; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const void *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::
            "r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

__global__ void __launch_bounds__(TMA_THREADS, 1)
stencil_tma_kernel(const InstDesc *__restrict__ inst, int ninst, const int *__restrict__ tprefix, int total_tiles,
                   int stage) {
    extern __shared__ unsigned char smem_dyn[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_dyn + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int4 info[2];          // (instance, x0, y0, flags) of the tile in each stage
    __shared__ float ssrc[2];         // source amplitude x stage forcing of that tile's instance
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    const int inb = stage_in(stage), outb = stage_out(stage);
    const uint32_t bytes = stage == 1 ? HALO_BYTES : STAGE_BYTES;

    auto issue = [&](int tile, int b) {           // thread 0: resolve the tile, start its copies
        const int ii = find_inst(tprefix, ninst, tile);
        const InstDesc &d = inst[ii];
        const int lt = tile - __ldg(tprefix + ii);
        const int tx = lt % d.tiles_x, ty = lt / d.tiles_x;
        const int x0 = tx * TILE_X, y0 = ty * TMA_TILE_Y;
        info[b] = make_int4(ii, x0, y0, (int)__ldg(d.tile_flags + lt));
        ssrc[b] = d.s_amp != 0.0 ? (float)(d.s_amp * stage_sigma<float>(d, stage)) : 0.f;
        unsigned char *dst = base + (size_t)b * STAGE_BYTES;
        mbar_arrive_expect_tx(&bar[b], bytes);
        tma_load_3d(dst, d.tmap[inb], &bar[b], x0 - HALO, y0 - HALO, 0);
        if (stage != 1) tma_load_3d(dst + HALO_BYTES, d.tmap[3], &bar[b], x0, y0, 0);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        if ((int)blockIdx.x < total_tiles) issue(blockIdx.x, 0);
        if ((int)(blockIdx.x + gridDim.x) < total_tiles) issue(blockIdx.x + gridDim.x, 1);
    }

    const int txi = tid % TMA_TX, tyi = tid / TMA_TX;
    const int cx0 = HALO + 4 * txi, ry0 = HALO + TMA_RY * tyi;   // halo-box coordinates of the first output
    const int lx0 = 4 * txi, ly0 = TMA_RY * tyi;                 // tile-local coordinates
    int k = 0;
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x, ++k) {
        const int b = k & 1;
        const uint32_t parity = (k >> 1) & 1;
        if (!mbar_wait_bounded(&bar[b], parity)) atomicExch(&abort_flag, 1);
        if (!abort_flag) {
            const int4 inf = info[b];
            const InstDesc &d = inst[inf.x];
            const int xt = inf.y, yt = inf.z;
            const uint32_t flags = (uint32_t)inf.w;
            const float *sp = (const float *)(base + (size_t)b * STAGE_BYTES);
            const float *su = sp + TB_X * TB_Y;
            const float *sv = su + TB_X * TB_Y;
            const float *qp = sv + TB_X * TB_Y;
            const float *qu = qp + TILE_X * TMA_TILE_Y;
            const float *qv = qu + TILE_X * TMA_TILE_Y;
            float *out = (float *)d.q[outb];
            const long long plane = d.plane;
            const int pitch = d.pitch, nx = d.nx, ny = d.ny;
            const float src = ssrc[b];
            const float ad = (float)(c_alpha[stage - 1] * d.dt);
            const float *gxs = (const float *)d.gx;
            const float *gys = (const float *)d.gy;
            const int gx0 = xt + lx0, gy0 = yt + ly0;
            if (flags == 0) {
                // interior: all outputs fluid, no band.  The stage update is
                // q - sum_j k_j (f_{+j} - f_{-j}) with k_j = alpha_k dt a_j / h.
                const double adh = c_alpha[stage - 1] * d.dt * d.inv_h;
                const float k1 = (float)(adh * 0.770882380518), k2 = (float)(adh * -0.166705904415),
                            k3 = (float)(adh * 0.020843142770);
                float dpy[TMA_RY][4], dvy[TMA_RY][4];
                {
                    float cp[TMA_RY + 6][4], cv[TMA_RY + 6][4];
#pragma unroll
                    for (int r = 0; r < TMA_RY + 6; ++r) {
                        const float4 a = *reinterpret_cast<const float4 *>(sp + (ry0 - 3 + r) * TB_X + cx0);
                        const float4 c = *reinterpret_cast<const float4 *>(sv + (ry0 - 3 + r) * TB_X + cx0);
                        cp[r][0] = a.x; cp[r][1] = a.y; cp[r][2] = a.z; cp[r][3] = a.w;
                        cv[r][0] = c.x; cv[r][1] = c.y; cv[r][2] = c.z; cv[r][3] = c.w;
                    }
#pragma unroll
                    for (int r = 0; r < TMA_RY; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            dpy[r][c] = k1 * (cp[r + 4][c] - cp[r + 2][c]) + k2 * (cp[r + 5][c] - cp[r + 1][c]) +
                                        k3 * (cp[r + 6][c] - cp[r][c]);
                            dvy[r][c] = k1 * (cv[r + 4][c] - cv[r + 2][c]) + k2 * (cv[r + 5][c] - cv[r + 1][c]) +
                                        k3 * (cv[r + 6][c] - cv[r][c]);
                        }
                }
#pragma unroll
                for (int r = 0; r < TMA_RY; ++r) {
                    float wp[12], wu[12];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const float4 a = *reinterpret_cast<const float4 *>(sp + (ry0 + r) * TB_X + cx0 - 4 + 4 * q);
                        const float4 c = *reinterpret_cast<const float4 *>(su + (ry0 + r) * TB_X + cx0 - 4 + 4 * q);
                        wp[4 * q] = a.x; wp[4 * q + 1] = a.y; wp[4 * q + 2] = a.z; wp[4 * q + 3] = a.w;
                        wu[4 * q] = c.x; wu[4 * q + 1] = c.y; wu[4 * q + 2] = c.z; wu[4 * q + 3] = c.w;
                    }
                    float4 n0, n1, n2;
                    if (stage == 1) {
                        n0 = make_float4(wp[4], wp[5], wp[6], wp[7]);
                        n1 = make_float4(wu[4], wu[5], wu[6], wu[7]);
                        n2 = *reinterpret_cast<const float4 *>(sv + (ry0 + r) * TB_X + cx0);
                    } else {
                        n0 = *reinterpret_cast<const float4 *>(qp + (ly0 + r) * TILE_X + lx0);
                        n1 = *reinterpret_cast<const float4 *>(qu + (ly0 + r) * TILE_X + lx0);
                        n2 = *reinterpret_cast<const float4 *>(qv + (ly0 + r) * TILE_X + lx0);
                    }
                    const float nn0[4] = {n0.x, n0.y, n0.z, n0.w}, nn1[4] = {n1.x, n1.y, n1.z, n1.w},
                                nn2[4] = {n2.x, n2.y, n2.z, n2.w};
                    const int gy = gy0 + r;
                    const float sy = src != 0.f ? ad * src * gys[gy] : 0.f;
                    float o0[4], o1[4], o2[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int q = 4 + c;
                        const float dpx = k1 * (wp[q + 1] - wp[q - 1]) + k2 * (wp[q + 2] - wp[q - 2]) + k3 * (wp[q + 3] - wp[q - 3]);
                        const float dux = k1 * (wu[q + 1] - wu[q - 1]) + k2 * (wu[q + 2] - wu[q - 2]) + k3 * (wu[q + 3] - wu[q - 3]);
                        float op = nn0[c] - (dux + dvy[r][c]);
                        if (src != 0.f) op += sy * gxs[gx0 + c];
                        o0[c] = op;
                        o1[c] = nn1[c] - dpx;
                        o2[c] = nn2[c] - dpy[r][c];
                    }
                    const long long o = (long long)gy * pitch + gx0;
                    *reinterpret_cast<float4 *>(out + o) = make_float4(o0[0], o0[1], o0[2], o0[3]);
                    *reinterpret_cast<float4 *>(out + plane + o) = make_float4(o1[0], o1[1], o1[2], o1[3]);
                    *reinterpret_cast<float4 *>(out + 2 * plane + o) = make_float4(o2[0], o2[1], o2[2], o2[3]);
                }
            } else {
                // band (one-sided + radiation), non-fluid nodes, ragged edges
                const float inv_h = (float)d.inv_h;
                const float half_inv_h = 0.5f * inv_h;
                for (int r = 0; r < TMA_RY; ++r) {
                    const int gy = gy0 + r, sr = ry0 + r;
                    if (gy >= ny) break;
                    for (int c = 0; c < 4; ++c) {
                        const int gx = gx0 + c, sc = cx0 + c;
                        if (gx >= nx) break;
                        const long long o = (long long)gy * pitch + gx;
                        const uint8_t kind = (flags & TILE_MIXED) ? __ldg(d.mask + o) : (uint8_t)1;
                        if (kind != 1) {
                            out[o] = 0.f; out[plane + o] = 0.f; out[2 * plane + o] = 0.f;
                            continue;
                        }
                        const bool band = gx < 3 || gx > nx - 4 || gy < 3 || gy > ny - 4;
                        auto fxp = [&](int q) { return sp[sr * TB_X + sc + q]; };
                        auto fxu = [&](int q) { return su[sr * TB_X + sc + q]; };
                        auto fyp = [&](int q) { return sp[(sr + q) * TB_X + sc]; };
                        auto fyv = [&](int q) { return sv[(sr + q) * TB_X + sc]; };
                        const float dpdx = deriv_general<float>(fxp, gx, nx, 0, inv_h);
                        const float dpdy = deriv_general<float>(fyp, gy, ny, 0, inv_h);
                        float rp, ru, rv;
                        if (!band) {
                            const float dudx = deriv_general<float>(fxu, gx, nx, 0, inv_h);
                            const float dvdy = deriv_general<float>(fyv, gy, ny, 0, inv_h);
                            rp = -(dudx + dvdy);
                            if (src != 0.f) rp += src * gxs[gx] * gys[gy];
                            ru = -dpdx;
                            rv = -dpdy;
                        } else {
                            auto fyu = [&](int q) { return su[(sr + q) * TB_X + sc]; };
                            auto fxv = [&](int q) { return sv[sr * TB_X + sc + q]; };
                            const float dudx = deriv_general<float>(fxu, gx, nx, 0, inv_h);
                            const float dudy = deriv_general<float>(fyu, gy, ny, 0, inv_h);
                            const float dvdx = deriv_general<float>(fxv, gx, nx, 0, inv_h);
                            const float dvdy = deriv_general<float>(fyv, gy, ny, 0, inv_h);
                            const float rx = float(gx) - (float)d.cx, ryy = float(gy) - (float)d.cy;
                            const float rho = sqrtf(rx * rx + ryy * ryy);
                            const float ct = rx / rho, st = ryy / rho;
                            const float q2 = half_inv_h / rho;
                            rp = -(ct * dpdx + st * dpdy + sp[sr * TB_X + sc] * q2);
                            ru = -(ct * dudx + st * dudy + su[sr * TB_X + sc] * q2);
                            rv = -(ct * dvdx + st * dvdy + sv[sr * TB_X + sc] * q2);
                        }
                        const int lq = (ly0 + r) * TILE_X + lx0 + c;
                        const float n0 = stage == 1 ? sp[sr * TB_X + sc] : qp[lq];
                        const float n1 = stage == 1 ? su[sr * TB_X + sc] : qu[lq];
                        const float n2 = stage == 1 ? sv[sr * TB_X + sc] : qv[lq];
                        out[o] = n0 + ad * rp;
                        out[plane + o] = n1 + ad * ru;
                        out[2 * plane + o] = n2 + ad * rv;
                    }
                }
            }
        }
        __syncthreads();                               // every thread is done with this stage
        if (abort_flag) {
            // a copy did not complete in time: flag the instance, let the other
            // stage's copy (if any) land, and leave
            if (tid == 0) {
                atomicOr((unsigned long long *)&inst[info[b].x].clock[2], 1ull);
                if (tile + (int)gridDim.x < total_tiles) mbar_wait_bounded(&bar[b ^ 1], ((k + 1) >> 1) & 1);
            }
            return;
        }
        const int nxt = tile + 2 * (int)gridDim.x;
        if (tid == 0 && nxt < total_tiles) issue(nxt, b);
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
    }
    __syncthreads();
    if (threadIdx.x == 0) d.clock[1] = rec + 1;
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

// ---------------------------------------------------------------- launchers
namespace {
template <typename T> size_t stencil_smem() { return (size_t)3 * SY * SX * sizeof(T); }

template <typename T> cudaError_t setup_stencil_attr() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(stencil_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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

cudaError_t prepare_kernels(int precision) {
    if (precision == 1) {
        static bool done = false;
        if (!done) {
            cudaError_t e = cudaFuncSetAttribute(stencil_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)TMA_SMEM);
            if (e != cudaSuccess) return e;
            done = true;
        }
        num_sms();
        return setup_stencil_attr<float>();
    }
    num_sms();
    return setup_stencil_attr<double>();
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
    const cuuint32_t halo_box[3] = {TB_X, TB_Y, 3};
    const cuuint32_t tile_box[3] = {TILE_X, TMA_TILE_Y, 3};
    for (int b = 0; b < 4; ++b) {
        CUresult r = enc(&maps[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, d.q[b < 3 ? b : 0], dims, strides,
                         b < 3 ? halo_box : tile_box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            err = "cuTensorMapEncodeTiled returned " + std::to_string((int)r);
            return false;
        }
    }
    return true;
}

cudaError_t launch_ghost(const BatchView &bv, int stage, cudaStream_t s) {
    const int blocks = bv.nchunks > 0 ? bv.nchunks : 1;
    if (bv.precision == 1)
        ghost_kernel<float><<<blocks, GHOST_THREADS, 0, s>>>(bv.inst, bv.ninst, bv.ghost_chunks, bv.nchunks, stage);
    else
        ghost_kernel<double><<<blocks, GHOST_THREADS, 0, s>>>(bv.inst, bv.ninst, bv.ghost_chunks, bv.nchunks, stage);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_stencil(const BatchView &bv, int stage, int persistent_ctas, cudaStream_t s) {
    cudaError_t e;
    if (bv.precision == 1 && bv.use_tma) {
        if (bv.total_tiles == 0) return cudaSuccess;
        const int grid = std::min(bv.total_tiles, persistent_ctas > 0 ? persistent_ctas : num_sms());
        stencil_tma_kernel<<<grid, TMA_THREADS, TMA_SMEM, s>>>(bv.inst, bv.ninst, bv.tile_prefix, bv.total_tiles, stage);
        count_launch();
        return cudaGetLastError();
    }
    const int grid = persistent_ctas > 0 ? std::min(persistent_ctas, bv.total_tiles) : bv.total_tiles;
    if (bv.precision == 1) {
        if ((e = setup_stencil_attr<float>()) != cudaSuccess) return e;
        stencil_kernel<float><<<grid, STENCIL_THREADS, stencil_smem<float>(), s>>>(bv.inst, bv.ninst, bv.tile_prefix,
                                                                                  bv.total_tiles, stage);
    } else {
        if ((e = setup_stencil_attr<double>()) != cudaSuccess) return e;
        stencil_kernel<double><<<grid, STENCIL_THREADS, stencil_smem<double>(), s>>>(bv.inst, bv.ninst, bv.tile_prefix,
                                                                                    bv.total_tiles, stage);
    }
    count_launch();
    return cudaGetLastError();
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

}  // namespace lee
