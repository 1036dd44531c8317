// lee_setup.cpp -- host set-up of one instance (FP64): mask, ghost set,
// boundary points, elliptical clouds, least-squares read-out rows by
// Householder QR, Lagrange extrapolation along the normal folded into four
// weight rows per ghost, ADE coefficients of the MSD wall, probe stencils and
// stencil-tile classification.
//
// Paper: Sec. 3.1 (Eqs. ns-rotation, ns-ellipse, ns-poly2d, ns-vandermonde,
// ns-LSQ, ns-readout, ns-ghost), Sec. 2.5 (MSD poles and residues), Sec. 3.2
// (what the stage kernels need per ghost point).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>

#include "lee_internal.h"
#include "../../include/lee.h"

namespace lee {

namespace {

constexpr int KMAX = 4;         // k = m = 4 (Sec. 3.1)
constexpr double RN = 8.0;      // R_n = 2k
constexpr double RT = 3.0;      // R_t = k/2 + 1
constexpr int MAXCLOUD = 160;

struct Setup {
    int nx, ny, per_x, per_y;
    double h, x0, y0;
    Geometry geo;
    double xi(int i) const { return x0 + i * h; }
    double yj(int j) const { return y0 + j * h; }
    // Fluid test of Sec. 3.1, in the canonical form shared with the written
    // definition: line (x - xw).n > 0, cylinder |x - c|^2 > r^2.
    bool fluid(double x, double y) const {
        if (geo.kind == 1) {
            const double nxl = -std::sin(geo.c), nyl = std::cos(geo.c);
            return (x - geo.a) * nxl + (y - geo.b) * nyl > 0.0;
        }
        if (geo.kind == 2) {
            const double dx = x - geo.a, dy = y - geo.b;
            return dx * dx + dy * dy > geo.c * geo.c;
        }
        return true;
    }
};

inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }

// Axis footprint [lo, hi] of the derivative at index i: the 7-point DRP in the
// interior (and on periodic axes), the one-sided 7-point DRP stencils on nodes
// 0..6 / n-7..n-1 in the three outer layers.
inline void axis_footprint(int i, int n, int per, int &lo, int &hi) {
    if (!per && i <= 2) { lo = 0; hi = 6; }
    else if (!per && i >= n - 3) { lo = n - 7; hi = n - 1; }
    else { lo = i - 3; hi = i + 3; }
}

// Extended precision for the least-squares and Lagrange factors; the weight
// rows are rounded to FP64 once, after they are combined.
using xr = long double;

// Householder QR of the column-scaled N x nm Vandermonde matrix and the
// read-out rows L_i = v(P_i)^T V^+ for P_i = (i, 0), i = 0..k.
// Returns false when |R_jj| spans more than 1e10 (rank deficient).
bool readout_rows(int N, const double *xp, const double *yp, int k, xr *L /* (k+1) x N */) {
    int ea[15], eb[15], nm = 0;
    for (int d = 0; d <= k; ++d)
        for (int a = d; a >= 0; --a) { ea[nm] = a; eb[nm] = d - a; ++nm; }
    if (N < nm) return false;
    auto pw = [](xr x, int e) { xr r = 1.0L; while (e-- > 0) r *= x; return r; };
    std::vector<xr> V((size_t)N * nm);               // column-major: V[j * N + e]
    xr scale[15];
    for (int j = 0; j < nm; ++j) {
        xr s2 = 0.0L;
        for (int e = 0; e < N; ++e) {
            xr v = pw(xp[e], ea[j]) * pw(yp[e], eb[j]);
            V[(size_t)j * N + e] = v;
            s2 += v * v;
        }
        scale[j] = s2 > 0.0L ? 1.0L / std::sqrt(s2) : 1.0L;
        for (int e = 0; e < N; ++e) V[(size_t)j * N + e] *= scale[j];
    }
    std::vector<xr> hv((size_t)N * nm, 0.0L);         // unit Householder vectors
    xr Rd[15];
    std::vector<xr> R((size_t)nm * nm, 0.0L);
    for (int j = 0; j < nm; ++j) {
        xr *col = &V[(size_t)j * N];
        xr nrm = 0.0L;
        for (int e = j; e < N; ++e) nrm += col[e] * col[e];
        nrm = std::sqrt(nrm);
        xr alpha = col[j] > 0 ? -nrm : nrm;
        xr *v = &hv[(size_t)j * N];
        for (int e = j; e < N; ++e) v[e] = col[e];
        v[j] -= alpha;
        xr vn = 0.0L;
        for (int e = j; e < N; ++e) vn += v[e] * v[e];
        vn = std::sqrt(vn);
        if (vn > 0.0L) for (int e = j; e < N; ++e) v[e] /= vn;
        // apply H_j = I - 2 v v^T to the remaining columns
        for (int jj = j; jj < nm; ++jj) {
            xr *cc = &V[(size_t)jj * N];
            xr dot = 0.0L;
            for (int e = j; e < N; ++e) dot += v[e] * cc[e];
            for (int e = j; e < N; ++e) cc[e] -= 2.0L * dot * v[e];
        }
        for (int i = 0; i <= j; ++i) R[(size_t)i * nm + j] = V[(size_t)j * N + i];
        Rd[j] = std::fabs(R[(size_t)j * nm + j]);
    }
    xr rmax = *std::max_element(Rd, Rd + nm), rmin = *std::min_element(Rd, Rd + nm);
    if (!(rmin > 1e-10L * rmax)) return false;
    std::vector<xr> y(N);
    for (int i = 0; i <= k; ++i) {
        xr z[15];
        // R^T z = D v(P_i), v(P_i) has x' = i, y' = 0
        for (int j = 0; j < nm; ++j) {
            xr rhs = (eb[j] == 0 ? pw((xr)i, ea[j]) : 0.0L) * scale[j];
            for (int l = 0; l < j; ++l) rhs -= R[(size_t)l * nm + j] * z[l];
            z[j] = rhs / R[(size_t)j * nm + j];
        }
        std::fill(y.begin(), y.end(), 0.0L);
        for (int j = 0; j < nm; ++j) y[j] = z[j];
        for (int j = nm - 1; j >= 0; --j) {            // y = H_0 ... H_{nm-1} [z; 0]
            const xr *v = &hv[(size_t)j * N];
            xr dot = 0.0L;
            for (int e = j; e < N; ++e) dot += v[e] * y[e];
            for (int e = j; e < N; ++e) y[e] -= 2.0L * dot * v[e];
        }
        for (int e = 0; e < N; ++e) L[(size_t)i * N + e] = y[e];
    }
    return true;
}

// Lagrange basis on nodes {first..m} (integers), value at s.
xr lag(int first, int m, int i, xr s) {
    xr v = 1.0L;
    for (int j = first; j <= m; ++j) if (j != i) v *= (s - j) / xr(i - j);
    return v;
}
// derivative at s of the same basis
xr lag_d(int first, int m, int i, xr s) {
    xr d = 0.0L;
    for (int k = first; k <= m; ++k) {
        if (k == i) continue;
        xr t = 1.0L / xr(i - k);
        for (int j = first; j <= m; ++j) if (j != i && j != k) t *= (s - j) / xr(i - j);
        d += t;
    }
    return d;
}

// Extrapolation factors along the normal for degree m, ghost at s = -r
// (s in units of h, s = 0 at the boundary point, s = i at P_i):
//  free       Q through (i, f_i), i = 0..m:          f_GP = sum_i dir[i] f_i
//  Dirichlet  Q through (0, g), (i, f_i), i >= 1:    f_GP = kd g + sum_{i>=1} dir[i] f_i
//  Neumann    Q'(0) = h g_n, Q(i) = f_i, i >= 1:     f_GP = kn h g_n + sum_{i>=1} neu[i] f_i
// The Neumann polynomial is written Q = sum_i f_i lh_i + beta w with lh the
// Lagrange basis on {1..m} and w(s) = prod_{i=1..m} (s - i), which vanishes
// on the nodes; Q'(0) = h g_n fixes beta.
void normal_factors(int m, double r, xr *dir, xr &kd, xr *neu, xr &kn) {
    const xr s = -(xr)r;
    for (int i = 0; i <= m; ++i) dir[i] = lag(0, m, i, s);
    kd = dir[0];
    xr w_s = 1.0L, w_d0 = 0.0L;
    for (int i = 1; i <= m; ++i) w_s *= (s - i);
    for (int k = 1; k <= m; ++k) {
        xr t = 1.0L;
        for (int j = 1; j <= m; ++j) if (j != k) t *= (0.0L - j);
        w_d0 += t;
    }
    kn = w_s / w_d0;
    neu[0] = 0.0L;
    for (int i = 1; i <= m; ++i) {
        xr lh = (m == 1) ? 1.0L : lag(1, m, i, s);
        xr lhd = (m == 1) ? 0.0L : lag_d(1, m, i, 0.0L);
        neu[i] = lh - lhd * kn;
    }
}

std::complex<double> rk4_poly(std::complex<double> z) {
    return 1.0 + z * (1.0 + z * (0.5 + z * (1.0 / 6.0 + z / 24.0)));
}

}  // namespace

void fill_stage_constants(double dt, double h, double kappa, float kf[4][8], double kd[4][8]) {
    static const double alpha[4] = {0.25, 1.0 / 3.0, 0.5, 1.0};       // 2N-storage Jameson scheme
    static const double a[3] = {0.770882380518, -0.166705904415, 0.020843142770};  // DRP, Sec. 2.2
    const double inv_h = 1.0 / h;
    for (int k = 0; k < 4; ++k) {
        const double ad = alpha[k] * dt, adh = ad * inv_h;
        double v[8] = {ad, adh * a[0], adh * a[1], adh * a[2], adh * kappa, inv_h, kappa * inv_h, 0.0};
        for (int i = 0; i < 8; ++i) {
            kd[k][i] = v[i];
            kf[k][i] = (float)v[i];
        }
    }
}

void stage_forcing_factors(double omega, double dt, double G_re[4], double G_im[4]) {
    // Stage k uses the moment of order j = 4 - k of sin(w t) over the step:
    // (j+1)!/dt^(j+1) int_0^dt (dt - s)^j / j! e^{i w s} ds
    //   = sum_{n >= 0} (i theta)^n (j+1)! / (j+n+1)!,  theta = w dt.
    const double th = omega * dt;
    for (int k = 1; k <= 4; ++k) {
        const int j = 4 - k;
        long double re = 0.0L, im = 0.0L, c = 1.0L, p = 1.0L;
        for (int n = 0; n < 400; ++n) {
            long double term = c * p;
            switch (n & 3) {
                case 0: re += term; break;
                case 1: im += term; break;
                case 2: re -= term; break;
                default: im -= term; break;
            }
            p *= (long double)th;
            c /= (long double)(j + n + 2);
            if (n > 4 && std::fabs((double)(c * p)) < 1e-22) break;
        }
        G_re[k - 1] = (double)re;
        G_im[k - 1] = (double)im;
    }
}

int build_plan(int nx, int ny, double h, double x0, double y0, int per_x, int per_y, double dt, int tile_w, int tile_h,
               int sponge_w, const Geometry &geo, const Impedance &imp, const std::vector<double> &probe_xy,
               Plan &P, std::string &err) {
    Setup S{nx, ny, per_x, per_y, h, x0, y0, geo};
    P = Plan();
    P.nx = nx; P.ny = ny;
    P.pitch = (nx + 31) / 32 * 32;
    P.tile_w = tile_w;
    P.tiles_x = (nx + tile_w - 1) / tile_w;
    P.tile_h = tile_h;
    P.tiles_y = (ny + tile_h - 1) / tile_h;
    const size_t n = (size_t)nx * ny;
    if (geo.kind == 2 && !(geo.c > 3.5 * h)) { err = "cylinder radius must exceed 3.5 h"; return LEE_ERR_GEOMETRY; }

    // ---- mask and ghost set (Sec. 3.1)
    P.kind.assign(n, 0);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) P.kind[(size_t)j * nx + i] = S.fluid(S.xi(i), S.yj(j)) ? 1 : 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (P.kind[(size_t)j * nx + i] != 1) continue;
            int lo, hi;
            axis_footprint(i, nx, per_x, lo, hi);
            for (int a = lo; a <= hi; ++a) { uint8_t &k = P.kind[(size_t)j * nx + wrapi(a, nx)]; if (!k) k = 2; }
            axis_footprint(j, ny, per_y, lo, hi);
            for (int b = lo; b <= hi; ++b) { uint8_t &k = P.kind[(size_t)wrapi(b, ny) * nx + i]; if (!k) k = 2; }
        }
    P.n_fluid = 0;
    for (size_t s = 0; s < n; ++s) {
        if (P.kind[s] == 2) P.g_target.push_back((int)s);
        P.n_fluid += P.kind[s] == 1;
    }
    const int ng = (int)P.g_target.size();
    if (ng > 0 && geo.kind == 0) { err = "ghost points without a wall"; return LEE_ERR_GEOMETRY; }

    // ---- per-ghost reconstruction
    struct GOut { int m, k; std::vector<int> idx; std::vector<double> w; double kp, ku, meta[5]; int status; };
    std::vector<GOut> out(ng);
#pragma omp parallel for schedule(dynamic, 8)
    for (int g = 0; g < ng; ++g) {
        GOut &G = out[g];
        G.status = 0;
        const int gi = P.g_target[g] % nx, gj = P.g_target[g] / nx;
        const double x = S.xi(gi), y = S.yj(gj);
        double nrx, nry, bpx, bpy, d;
        if (geo.kind == 2) {
            const double gx = x - geo.a, gy = y - geo.b;
            const double rho = std::sqrt(gx * gx + gy * gy);
            nrx = gx / rho; nry = gy / rho;
            bpx = geo.a + geo.c * nrx; bpy = geo.b + geo.c * nry;
            d = geo.c - rho;
        } else {
            nrx = -std::sin(geo.c); nry = std::cos(geo.c);
            const double phi = (x - geo.a) * nrx + (y - geo.b) * nry;
            d = -phi;
            bpx = x + d * nrx; bpy = y + d * nry;
        }
        const double r = d / h;
        G.meta[0] = bpx; G.meta[1] = bpy; G.meta[2] = nrx; G.meta[3] = nry; G.meta[4] = r;
        // elliptical cloud (Eq. ns-ellipse), rotated reduced frame (Eq. ns-rotation)
        double xp[MAXCLOUD], yp[MAXCLOUD];
        int N = 0;
        const int ic = (int)std::floor((bpx - x0) / h), jc = (int)std::floor((bpy - y0) / h);
        for (int jj = jc - 10; jj <= jc + 10 && G.status == 0; ++jj) {
            if (!per_y && (jj < 0 || jj >= ny)) continue;
            for (int ii = ic - 10; ii <= ic + 10; ++ii) {
                if (!per_x && (ii < 0 || ii >= nx)) continue;
                const int s = wrapi(jj, ny) * nx + wrapi(ii, nx);
                if (P.kind[s] != 1) continue;
                const double ddx = S.xi(ii) - bpx, ddy = S.yj(jj) - bpy;
                const double xr = (nrx * ddx + nry * ddy) / h;
                const double yr = (-nry * ddx + nrx * ddy) / h;
                if ((xr * xr) / (RN * RN) + (yr * yr) / (RT * RT) <= 1.0) {
                    if (N == MAXCLOUD) { G.status = LEE_ERR_GEOMETRY; break; }
                    G.idx.push_back(s); xp[N] = xr; yp[N] = yr; ++N;
                }
            }
        }
        if (G.status) continue;
        std::vector<xr> L((size_t)(KMAX + 1) * (N > 0 ? N : 1));
        int m = KMAX;
        while (m >= 1 && !readout_rows(N, xp, yp, m, L.data())) --m;
        G.k = m >= 1 ? m : 0;
        if (m < 1) {
            // no plane through the cloud (its nodes on one line, where a steep
            // wall leaves the box): constant fit = cloud mean, read out at
            // P_0 and P_1, with a linear extrapolation along the normal
            if (N < 1) { G.status = LEE_ERR_RANK; continue; }
            for (int e = 0; e < N; ++e) L[e] = L[(size_t)N + e] = 1.0L / (xr)N;
            m = 1;
        }
        G.m = m;
        xr dir[KMAX + 1], neu[KMAX + 1], kd, kn;
        normal_factors(m, r, dir, kd, neu, kn);
        G.kp = (double)(kn * (xr)h);   // multiplies dp/dn at BP
        G.ku = (double)kd;             // multiplies w = u.n at BP
        G.w.assign((size_t)4 * N, 0.0);
        for (int e = 0; e < N; ++e) {
            xr l0 = L[e], wp = 0.0L, wd = 0.0L, wf = dir[0] * L[e];
            for (int i = 1; i <= m; ++i) {
                const xr li = L[(size_t)i * N + e];
                wp += neu[i] * li;
                wd += dir[i] * li;
                wf += dir[i] * li;
            }
            G.w[4 * e + 0] = (double)l0; G.w[4 * e + 1] = (double)wp;
            G.w[4 * e + 2] = (double)wd; G.w[4 * e + 3] = (double)wf;
        }
    }
    P.g_start.assign(ng + 1, 0);
    P.g_meta.resize((size_t)5 * ng);
    P.g_m.resize(ng);
    P.g_kappa.resize((size_t)2 * ng);
    for (int g = 0; g < ng; ++g) {
        if (out[g].status) {
            char b[160];
            snprintf(b, sizeof b, "ghost %d at node %d: %s", g, P.g_target[g],
                     out[g].status == LEE_ERR_RANK ? "cloud holds no fluid node" : "cloud too large");
            err = b;
            return out[g].status;
        }
        P.g_start[g + 1] = P.g_start[g] + (int)out[g].idx.size();
        for (int q = 0; q < 5; ++q) P.g_meta[(size_t)5 * g + q] = out[g].meta[q];
        P.g_m[g] = out[g].m;
        P.n_reduced += out[g].k < KMAX;
        P.g_kappa[2 * g] = out[g].kp;
        P.g_kappa[2 * g + 1] = out[g].ku;
    }
    P.e_idx.reserve(P.g_start[ng]);
    P.e_w.reserve((size_t)4 * P.g_start[ng]);
    for (int g = 0; g < ng; ++g) {
        P.e_idx.insert(P.e_idx.end(), out[g].idx.begin(), out[g].idx.end());
        P.e_w.insert(P.e_w.end(), out[g].w.begin(), out[g].w.end());
    }

    // ---- ADE of the MSD wall (Sec. 2.5), or of a rational admittance (Sec. 2.3)
    if (imp.rational()) {
        // Eq. ADEgeneral as X' = A X + b p_BP, u_n = c . X (Eq. unGeneral),
        // A block diagonal: one 1 x 1 block per real pole, one rotation block
        // [[al, -be], [be, al]] per pair
        const int ns = imp.nreal + 2 * imp.npair;
        P.regime = 4;
        P.ns = ns;
        P.ade_coef.assign((size_t)ns * ns + 2 * ns, 0.0);
        double *A = P.ade_coef.data(), *b = A + (size_t)ns * ns, *c = b + ns;
        double amp = 0.0;
        for (int k = 0; k < imp.nreal; ++k) {
            if (!(imp.lam[k] < 0)) { err = "rational admittance: real poles must be negative"; return LEE_ERR_ARG; }
            A[(size_t)k * ns + k] = imp.lam[k];
            b[k] = 1.0;
            c[k] = imp.A[k];
            amp = std::max(amp, std::abs(rk4_poly(std::complex<double>(imp.lam[k] * dt, 0.0))));
        }
        for (int k = 0; k < imp.npair; ++k) {
            if (!(imp.al[k] < 0 && imp.be[k] > 0)) {
                err = "rational admittance: pairs need alpha < 0 < beta";
                return LEE_ERR_ARG;
            }
            const int i = imp.nreal + 2 * k;
            A[(size_t)i * ns + i] = imp.al[k];
            A[(size_t)i * ns + i + 1] = -imp.be[k];
            A[(size_t)(i + 1) * ns + i] = imp.be[k];
            A[(size_t)(i + 1) * ns + i + 1] = imp.al[k];
            b[i] = 1.0;
            c[i] = 2.0 * imp.B[k];
            c[i + 1] = -2.0 * imp.C[k];
            amp = std::max(amp, std::abs(rk4_poly(std::complex<double>(imp.al[k], imp.be[k]) * dt)));
        }
        P.ade_amp = amp;
        if (ns == 2) {          // the two-state kernel path takes it like an MSD wall
            for (int q = 0; q < 4; ++q) P.A[q] = A[q];
            P.b[0] = b[0]; P.b[1] = b[1]; P.c[0] = c[0]; P.c[1] = c[1];
        }
    } else if (imp.rigid) {
        P.regime = 0;
        P.ade_amp = 0.0;
    } else {
        const double R = imp.R, M = imp.M, K = imp.K;
        if (!(R > 0 && M > 0 && K > 0)) { err = "impedance needs R, M, K > 0"; return LEE_ERR_ARG; }
        const double a = R / (2.0 * M);
        const double disc = a * a - K / M;
        std::complex<double> p1, p2;
        if (std::fabs(disc) <= 1e-10 * a * a) {
            // double pole lam = -a: Y = (1/M)(1/(s - lam) + lam/(s - lam)^2)
            const double lam = -a;
            P.regime = 3;
            P.A[0] = lam; P.A[1] = 0; P.A[2] = 1; P.A[3] = lam;
            P.b[0] = 1; P.b[1] = 0;
            P.c[0] = 1.0 / M; P.c[1] = lam / M;
            p1 = p2 = lam;
        } else if (disc < 0) {
            // s1 = -a + i beta, residue s1 / (M (s1 - s2)) = 1/(2M) + i a / (2 beta M)
            const double beta = std::sqrt(-disc);
            P.regime = 1;
            P.A[0] = -a; P.A[1] = -beta; P.A[2] = beta; P.A[3] = -a;
            P.b[0] = 1; P.b[1] = 0;
            P.c[0] = 1.0 / M;                     // 2 B1
            P.c[1] = -a / (beta * M);             // -2 C1
            p1 = {-a, beta}; p2 = {-a, -beta};
        } else {
            // two real poles; the larger-magnitude one first, the other from
            // the product l1 l2 = K / M (no cancellation)
            const double l2 = -a - std::sqrt(disc);
            const double l1 = (K / M) / l2;
            P.regime = 2;
            P.A[0] = l1; P.A[1] = 0; P.A[2] = 0; P.A[3] = l2;
            P.b[0] = 1; P.b[1] = 1;
            P.c[0] = l1 / (M * (l1 - l2));
            P.c[1] = l2 / (M * (l2 - l1));
            p1 = l1; p2 = l2;
        }
        P.ade_amp = std::max(std::abs(rk4_poly(p1 * dt)), std::abs(rk4_poly(p2 * dt)));
    }

    // the two-state forms in the dense layout as well, so that a batch whose
    // ghost kernel runs the general ADE (some member has ns != 2) takes them too
    if (P.ade_coef.empty())
        P.ade_coef = {P.A[0], P.A[1], P.A[2], P.A[3], P.b[0], P.b[1], P.c[0], P.c[1]};

    // ---- probes: 4 x 4 Lagrange (degree 3), else nearest fluid node
    const int np = (int)probe_xy.size() / 2;
    P.p_idx.assign((size_t)16 * np, 0);
    P.p_w.assign((size_t)16 * np, 0.0);
    for (int p = 0; p < np; ++p) {
        const double fx = (probe_xy[2 * p] - x0) / h, fy = (probe_xy[2 * p + 1] - y0) / h;
        const int i0 = (int)std::floor(fx) - 1, j0 = (int)std::floor(fy) - 1;
        bool ok = i0 >= 0 && j0 >= 0 && i0 + 3 < nx && j0 + 3 < ny;
        for (int b = 0; ok && b < 4; ++b)
            for (int a = 0; a < 4; ++a) ok = ok && P.kind[(size_t)(j0 + b) * nx + i0 + a] == 1;
        if (ok) {
            const double xi = fx - i0, eta = fy - j0;
            for (int b = 0; b < 4; ++b)
                for (int a = 0; a < 4; ++a) {
                    P.p_idx[16 * p + 4 * b + a] = (j0 + b) * nx + i0 + a;
                    P.p_w[16 * p + 4 * b + a] = (double)(lag(0, 3, a, xi) * lag(0, 3, b, eta));
                }
        } else {
            const int i = (int)std::floor(fx + 0.5), j = (int)std::floor(fy + 0.5);
            if (i >= 0 && j >= 0 && i < nx && j < ny && P.kind[(size_t)j * nx + i] == 1) {
                P.p_idx[16 * p] = j * nx + i;
                P.p_w[16 * p] = 1.0;
            }
        }
    }

    // ---- stencil tiles: band / mixed flags
    P.tile_flags.assign((size_t)P.tiles_x * P.tiles_y, 0u);
    for (int ty = 0; ty < P.tiles_y; ++ty)
        for (int tx = 0; tx < P.tiles_x; ++tx) {
            uint32_t f = 0;
            const int xa = tx * tile_w, xb = xa + tile_w, ya = ty * tile_h, yb = ya + tile_h;
            if (!per_x && (xa < 3 || xb > nx - 3)) f |= TILE_BAND;
            if (!per_y && (ya < 3 || yb > ny - 3)) f |= TILE_BAND;
            if (per_x || per_y) f |= TILE_BAND;        // wrapped halos take the general path
            if (sponge_w > 0 &&
                ((!per_x && (xa < sponge_w || xb > nx - sponge_w)) || (!per_y && (ya < sponge_w || yb > ny - sponge_w))))
                f |= TILE_SPONGE;
            if (xb > nx || yb > ny) f |= TILE_MIXED;
            for (int j = ya; j < std::min(yb, ny) && !(f & TILE_MIXED); ++j)
                for (int i = xa; i < std::min(xb, nx); ++i)
                    if (P.kind[(size_t)j * nx + i] != 1) { f |= TILE_MIXED; break; }
            if ((f & TILE_BAND) && !per_x && !per_y && nx >= 7 && ny >= 7) {
                // every band node of the tile, and every node of its x and y
                // windows (7 nodes, one-sided near an edge), is fluid
                bool fluid = true;
                auto ok = [&](int i, int j) { return P.kind[(size_t)j * nx + i] == 1; };
                for (int j = ya; j < std::min(yb, ny) && fluid; ++j)
                    for (int i = xa; i < std::min(xb, nx) && fluid; ++i) {
                        if (!(j < 3 || j > ny - 4 || i < 3 || i > nx - 4)) continue;
                        const int sx = std::min(std::max(i - 3, 0), nx - 7), sy = std::min(std::max(j - 3, 0), ny - 7);
                        for (int k = 0; k < 7 && fluid; ++k) fluid = ok(sx + k, j) && ok(i, sy + k);
                    }
                if (fluid) f |= TILE_BAND_FLUID;
            }
            bool inert = true;                 // solid (kind 0) everywhere: no fluid node, no ghost
            for (int j = ya; j < std::min(yb, ny) && inert; ++j)
                for (int i = xa; i < std::min(xb, nx) && inert; ++i) inert = P.kind[(size_t)j * nx + i] == 0;
            if (inert) f |= TILE_INERT;
            P.tile_flags[(size_t)ty * P.tiles_x + tx] = f;
        }
    return LEE_OK;
}

}  // namespace lee
