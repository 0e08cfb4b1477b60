// tlb_device.cuh -- device code of the ternary free-energy ELBM step
// (arXiv:1904.06881, Sec. II-IV) for sm_103a.  Included by one translation
// unit per lattice (tlb_d2q9.cu, tlb_d3q27.cu).
//
// Data layout in HBM (one lattice of N nodes, x fastest, periodic):
//   f  : float[Q][N]  pre-collision populations stored as f_i - w_i
//   g  : float[Q][N], or (reduced precision) g_0 as float[N] followed by the
//        moving populations as half[Q-1][N] scaled by 16
//   rho, phi : float[N] moments of the current state, written by the moments
//              kernel (ghost values are computed in shared memory by the step
//              kernels; only the auxiliary-output and allocation-free paths
//              write them to these arrays)
//   type : uint8[N]  node flags (TLB_SOLID, TLB_FIRST, TLB_GHOST, TLB_NEAR, wall axes)
// One step, through a tile -> lattice table (the same kernels for one lattice
// and for a batch):
//   D2Q9  : step_batch_kernel alone -- rho, phi of the tile + halo 2 summed
//           from the populations, ghost layer, stencils, chemical potentials,
//           pressure tensor (halo 1), force with wall rules, ELBM collision of
//           f (entropic alpha), LBGK of g, push streaming with halfway
//           bounce-back;
//   D3Q27 : moments_batch_kernel (rho = 1 + sum_i f~_i, phi = sum_i g_i), then
//           step_batch_kernel as above with rho, phi read from the moments.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "tlb_internal.h"

namespace tlb {

// ---------------------------------------------------------------------------
// Lattice tables (own enumeration: rest, then +c/-c pairs).
// ---------------------------------------------------------------------------
template <int D>
struct Lat;

template <>
struct Lat<2> {
    static constexpr int Q = 9;
    static constexpr int NPOS = 4;
    __host__ __device__ static constexpr int pos(int k, int a)
    {
        // positive directions: (1,0) (0,1) (1,1) (1,-1)
        return a == 2 ? 0 : (k == 0 ? (a == 0 ? 1 : 0) : k == 1 ? (a == 0 ? 0 : 1) : k == 2 ? 1 : (a == 0 ? 1 : -1));
    }
};

template <>
struct Lat<3> {
    static constexpr int Q = 27;
    static constexpr int NPOS = 13;
    __host__ __device__ static constexpr int pos(int k, int a)
    {
        // (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)
        // (1,1,1) (1,1,-1) (1,-1,1) (1,-1,-1)
        constexpr int t[13][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1},
                                  {0, 1, 1}, {0, 1, -1}, {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
        return t[k][a];
    }
};

template <int D>
__host__ __device__ constexpr int cc(int i, int a)
{
    return i == 0 ? 0 : ((i - 1) % 2 == 0 ? Lat<D>::pos((i - 1) / 2, a) : -Lat<D>::pos((i - 1) / 2, a));
}

template <int D>
__host__ __device__ constexpr int opp(int i)
{
    return i == 0 ? 0 : ((i - 1) % 2 == 0 ? i + 1 : i - 1);
}

// weights: product of D1Q3 weights 2/3 (c = 0) and 1/6 (c = +-1)
template <int D>
__host__ __device__ constexpr float wt(int i)
{
    float w = 1.0f;
    for (int a = 0; a < D; ++a) w *= (cc<D>(i, a) == 0) ? (2.0f / 3.0f) : (1.0f / 6.0f);
    return w;
}

// ---------------------------------------------------------------------------
// Geometry helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapi(int v, int n)
{
    v %= n;
    return v < 0 ? v + n : v;
}

// Bounds-checked builds (-DTLB_BOUNDS_CHECK): every node index the kernels
// compute passes through chk_node; one outside [0, N) sets this translation
// unit's error word (read by Launch<D>::bounds_errors) and is replaced by 0,
// so the access stays inside the array.  Without the flag chk_node is the
// identity.
#ifdef TLB_BOUNDS_CHECK
static __device__ unsigned g_bounds_error;
__device__ __forceinline__ long long chk_node(long long n, const DevParams &p)
{
    if (n < 0 || n >= p.N) {
        atomicOr(&g_bounds_error, 1u);
        return 0;
    }
    return n;
}
#else
__device__ __forceinline__ long long chk_node(long long n, const DevParams &) { return n; }
#endif

__device__ __forceinline__ long long node_of(const DevParams &p, int x, int y, int z)
{
    return chk_node(
        (long long)wrapi(x, p.nx) + (long long)p.nx * ((long long)wrapi(y, p.ny) + (long long)p.ny * wrapi(z, p.nz)), p);
}

// ---------------------------------------------------------------------------
// Thermodynamics (Sec. II.A-B), FP32
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gpoly(float x) { return x * (x - 0.5f) * (x - 1.0f); }

struct Bulk {
    float murB, mupB, p0;
};

// Bulk chemical potentials and pressure at (rho, phi): Eqs. BulkEnergy,
// bulkchempotrho (lambda_2 term with the sign of the derivative of
// Eq. BulkEnergy), bulkchempotphi, bulkpressure, with the Carnahan-Starling
// Psi of Eq. PsiEOS and its printed derivative.
__device__ __forceinline__ Bulk bulk_terms(const DevParams &p, float rho, float phi)
{
    float C1 = (rho - p.rho_l) * p.inv_rgl;            // (rho - rho_l)/(rho_g - rho_l)
    float C2 = 0.5f * (1.0f + phi * p.inv_chi - C1);
    float C3 = 0.5f * (1.0f - phi * p.inv_chi - C1);
    float br = p.b * rho;
    float psi, dpsi;
    if (p.eos == 0) {
        // Carnahan-Starling, Eq. PsiEOS and its printed derivative
        float q = br - 4.0f;
        float lr = __logf(rho);
        psi = rho * (p.C - p.a * rho - 8.0f * p.RT * (br - 6.0f) / (q * q) + p.RT * lr);
        dpsi = p.C - 2.0f * p.a * rho + p.RT * (1.0f + lr) + 16.0f * p.RT * (br - 12.0f) / (q * q * q);
    } else {
        // van der Waals: Psi = rho (C - a rho + RT ln(rho/(1 - b rho)));
        // Peng-Robinson adds - a A/(2 sqrt2 b) ln((b rho + sqrt2 - 1)/(sqrt2 + 1 - b rho))
        // inside the bracket in place of - a rho (a A: p.aA)
        const float om = 1.0f - br;
        const float lg = __logf(rho / om);
        if (p.eos == 1) {
            psi = rho * (p.C - p.a * rho + p.RT * lg);
            dpsi = p.C - 2.0f * p.a * rho + p.RT * lg + p.RT / om;
        } else {
            const float k = p.aA * (0.35355339f / p.b);      // a A / (2 sqrt2 b)
            const float L = __logf((br + 0.41421356f) / (2.41421356f - br));
            psi = rho * (p.C + p.RT * lg - k * L);
            dpsi = p.C + p.RT * lg + p.RT / om - k * L - p.aA * rho / (1.0f + 2.0f * br - br * br);
        }
    }
    float g2 = gpoly(C2), g3 = gpoly(C3);
    float fb = 0.5f * p.lam1 * (psi - p.Psi0) + 0.5f * p.lam2 * C2 * C2 * (1.0f - C2) * (1.0f - C2) +
               0.5f * p.lam3 * C3 * C3 * (1.0f - C3) * (1.0f - C3);
    Bulk r;
    r.murB = 0.5f * p.lam1 * dpsi + (p.lam2 * g2 + p.lam3 * g3) * p.inv_drho;
    r.mupB = (p.lam2 * g2 - p.lam3 * g3) * p.inv_chi;
    r.p0 = rho * r.murB + phi * r.mupB - fb;
    return r;
}

// ELBM beta of a node: the fluid's beta, or with per-component viscosities
// the beta of the concentration-weighted mean viscosity (concentrations
// clipped to [0, 1]), nu = (1/beta - 1)/6.
__device__ __forceinline__ float local_beta(const DevParams &p, float rho, float phi)
{
    if (!p.nu_on) return p.beta;
    const float C1 = (rho - p.rho_l) * p.inv_rgl;
    const float C2 = 0.5f * (1.0f + phi * p.inv_chi - C1), C3 = 0.5f * (1.0f - phi * p.inv_chi - C1);
    const float c1 = fminf(fmaxf(C1, 0.f), 1.f), c2 = fminf(fmaxf(C2, 0.f), 1.f), c3 = fminf(fmaxf(C3, 0.f), 1.f);
    const float nu = (c1 * p.nu[0] + c2 * p.nu[1] + c3 * p.nu[2]) / (c1 + c2 + c3);
    return 1.0f / (6.0f * nu + 1.0f);
}

// ---------------------------------------------------------------------------
// Product-form equilibrium (Eqs. eqrho, A, B): per axis the three D1Q3
// factors w(c) A(u) B(u)^c, c = 0, +1, -1.
// ---------------------------------------------------------------------------
struct Fac {
    float f0, fp, fm;
};

__device__ __forceinline__ Fac eq_factors(float u)
{
    float s = sqrtf(1.0f + 3.0f * u * u);
    float A = 2.0f - s;
    float B = (2.0f * u + s) / (1.0f - u);
    Fac r;
    r.f0 = (2.0f / 3.0f) * A;
    r.fp = (1.0f / 6.0f) * A * B;
    r.fm = (1.0f / 6.0f) * A / B;
    return r;
}

__device__ __forceinline__ float fac_of(const Fac &f, int c) { return c == 0 ? f.f0 : (c > 0 ? f.fp : f.fm); }

// phi(y) = (1 + y) ln(1 + y) - y given l = ln(1 + y), accurate for small |y|
// (series y^2/2 - y^3/6 + ...)
__device__ __forceinline__ float phi_ent(float y, float l)
{
    if (fabsf(y) < 1e-2f) return y * y * (0.5f + y * (-1.0f / 6.0f + y * (1.0f / 12.0f - y * (1.0f / 20.0f))));
    return (1.0f + y) * l - y;
}

// Entropic alpha: the non-trivial root of H(f' + alpha D) = H(f')
// (Eq. EntropyEquation) with D = f^eq(u) - f = f^eq(u + du) - f'.  With
// x_i = D_i / f'_i, and because D carries no mass or momentum while
// ln(f^eq_i(u+du)/w_i) is affine in c_i,
//   h(alpha) = sum_i f'_i [ phi(alpha x_i) - alpha x_i ln(1 + x_i) ],
//   h'(alpha) = sum_i f'_i x_i [ ln(1 + alpha x_i) - ln(1 + x_i) ],
//   h''(alpha) = sum_i f'_i x_i^2 / (1 + alpha x_i),
// which involves no difference of O(1) entropies.  Expanding h/alpha in x
// with the moments a_k = sum_i f'_i x_i^k (a_1 = 0), b_k = a_k / a_2, and
// solving alpha = 2 + e1 + ... + e5 order by order gives
//   e1 = b3 / 3,  e2 = 2 (2 b3^2 - 3 b4) / 9,
//   e3 = (297 b5 - 420 b3 b4 + 170 b3^3) / 270,
//   e4 = (1026 b3 b5 + 540 b4^2 - 702 b6 - 1305 b3^2 b4 + 380 b3^4) / 405,
//   e5 = (15390 b7 - 23184 b3 b6 - 24570 b4 b5 + 30114 b3^2 b5 + 31080 b3 b4^2
//         - 36295 b3^3 b4 + 8260 b3^5) / 5670,
// used as is up to max|x| = ALPHA_SERIES_MAX = 0.1 (against the exact FP64
// root of random D2Q9 and D3Q27 states on the equilibrium manifold its
// truncation error is below 8e-8 at max|x| = 0.07 and 7e-7 at 0.1, about three
// units in the last place of alpha, and moves f by less than 4e-8 of itself)
// and as the start of Halley's method (third order, from h, h', h''),
// bracketed by [1, alpha_max), above it (nodes at the interface).
// FPA: accessor of f'_i.
constexpr float ALPHA_SERIES_MAX = 0.1f;
template <int Q, class FPA>
__device__ __forceinline__ float alpha_series_a(const FPA &fp, const float (&x)[Q])
{
    float a2 = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f, a6 = 0.f, a7 = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const float x2 = x[i] * x[i];
        const float fx2 = fp(i) * x2, fx4 = fx2 * x2;
        a2 += fx2;
        a3 += fx2 * x[i];
        a4 += fx4;
        a5 += fx4 * x[i];
        a6 += fx4 * x2;
        a7 += fx4 * x2 * x[i];
    }
    if (!(a2 > 0.f)) return 2.0f;
    const float r = 1.0f / a2;
    const float b3 = a3 * r, b4 = a4 * r, b5 = a5 * r, b6 = a6 * r, b7 = a7 * r;
    const float b33 = b3 * b3;
    const float e1 = b3 * (1.0f / 3.0f);
    const float e2 = (2.0f / 9.0f) * (2.0f * b33 - 3.0f * b4);
    const float e3 = (297.0f * b5 - 420.0f * b3 * b4 + 170.0f * b33 * b3) * (1.0f / 270.0f);
    const float e4 = (1026.0f * b3 * b5 + 540.0f * b4 * b4 - 702.0f * b6 - 1305.0f * b33 * b4 + 380.0f * b33 * b33) *
                     (1.0f / 405.0f);
    const float e5 = (15390.0f * b7 - 23184.0f * b3 * b6 - 24570.0f * b4 * b5 + 30114.0f * b33 * b5 +
                      31080.0f * b3 * b4 * b4 - 36295.0f * b33 * b3 * b4 + 8260.0f * b33 * b33 * b3) *
                     (1.0f / 5670.0f);
    return 2.0f + e1 + e2 + e3 + e4 + e5;
}

template <int Q>
struct RegPop {
    const float (&v)[Q];
    __device__ __forceinline__ float operator()(int i) const { return v[i]; }
};

template <int Q>
__device__ __forceinline__ float alpha_series(const float (&fp)[Q], const float (&x)[Q])
{
    return alpha_series_a<Q>(RegPop<Q>{fp}, x);
}

// Root of h in (1, alpha_max) from the start al.  h(1) < 0 always; when h is
// still negative at the positivity bound there is no root below it and the
// bound is returned.  h is evaluated at the bound only when an update would
// cross it.  An update of at most 1e-3 alpha is applied and ends the
// iteration: the third-order convergence leaves an error of order 1e-9
// alpha, below the FP32 evaluation noise of h (about 1e-6 alpha at
// max|x| = 0.5).
template <int Q, class FPA>
__device__ __forceinline__ float alpha_newton_a(const FPA &fp, const float (&x)[Q], float amax, float al)
{
    float L[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) L[i] = log1pf(x[i]);
    const float bound = amax * (1.0f - 1e-6f);
    float lo = 1.0f, hi = bound;
    bool probed = false;
    if (!(al > lo && al < hi)) al = 0.5f * (lo + hi);
    float a = al;
#pragma unroll 1
    for (int it = 0; it < 20; ++it) {
        // the terms of h, h', h'' are independent: unrolled for instruction-level parallelism
        float h = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float y = a * x[i];
            const float ly = log1pf(y);
            const float f = fp(i);
            h += f * (phi_ent(y, ly) - y * L[i]);
            d1 += f * x[i] * (ly - L[i]);
            d2 += f * x[i] * x[i] / (1.0f + y);
        }
        if (a == bound) {
            if (h < 0.f) return bound;        // no root below the positivity bound
            probed = true;                    // the bound brackets the root: bisect
            a = 0.5f * (lo + hi);
            continue;
        }
        al = a;
        if (h > 0.f) hi = al; else lo = al;
        float nxt;
        if (d1 > 0.f) {
            const float s = h / d1;
            const float step = s / (1.0f - 0.5f * s * d2 / d1);   // Halley's update
            if (fabsf(step) <= 1e-3f * al) return fminf(al - step, bound);
            nxt = al - step;
            if (!(nxt > lo && nxt < hi)) {
                if (nxt >= hi && hi == bound && !probed) {
                    a = bound;
                    continue;
                }
                nxt = 0.5f * (lo + hi);
            }
        } else {
            nxt = 0.5f * (lo + hi);
        }
        if (hi - lo <= 2e-6f * hi) return nxt;
        a = nxt;
    }
    return a;
}

template <int Q>
__device__ __forceinline__ float alpha_newton(const float (&fp)[Q], const float (&x)[Q], float amax, float al)
{
    return alpha_newton_a<Q>(RegPop<Q>{fp}, x, amax, al);
}

// ---------------------------------------------------------------------------
// Ghost layer (Sec. IV): one fluid-facing direction of a ghost node.
// ---------------------------------------------------------------------------
// A node accessor answers, for a node given by coordinates that are not
// wrapped (they may lie a few nodes outside the lattice), whether it is a
// fluid node and, if so, its moments (rho, phi).
//
// NodesGlobal: node flags and the moment arrays the moments kernel writes.
struct NodesGlobal {
    const DevParams &p;
    const uint8_t *type;
    const float *rho, *phi;
    __device__ __forceinline__ bool get(int x, int y, int z, float2 &m) const
    {
        const long long n = node_of(p, x, y, z);
        if (type[n] & TLB_SOLID) return false;
        m = make_float2(rho[n], phi[n]);
        return true;
    }
};

// The ghost value of one fluid-facing axis direction: (yx, yy, yz) is the
// first fluid node along `axis`, m1 its moments; `acc` a node accessor.
template <int D, class A>
__device__ void ghost_axis(const DevParams &p, const A &acc, int yx, int yy, int yz, int axis, float2 m1, float &gr,
                           float &gp)
{
    // Coordinates are kept in scalars (an array indexed by the run-time axis
    // would live in local memory): the in-plane axes are t0 = first axis other
    // than `axis`, t1 = the second (3D), as unit offsets (ux, uy, uz), (vx, vy, vz).
    const float r1 = m1.x, p1 = m1.y;
    if (p.wetting == TLB_WET_FORCE) { gr = r1; gp = p1; return; }
    const int t0 = axis == 0 ? 1 : 0, t1 = axis == 2 ? 1 : 2;
    const int ux = t0 == 0, uy = t0 == 1, uz = 0;
    const int vx = 0, vy = (D == 3 && t1 == 1), vz = (D == 3 && t1 == 2);
    // in-plane central (one-sided next to solid) differences of rho, phi
    auto diff = [&](int ox, int oy, int oz, float &dr, float &dp) {
        float2 a, b;
        const bool fp_ = acc.get(yx + ox, yy + oy, yz + oz, a), fm = acc.get(yx - ox, yy - oy, yz - oz, b);
        dr = 0.f;
        dp = 0.f;
        if (fp_ && fm) {
            dr = 0.5f * (a.x - b.x);
            dp = 0.5f * (a.y - b.y);
        } else if (fp_) {
            dr = a.x - r1;
            dp = a.y - p1;
        } else if (fm) {
            dr = r1 - b.x;
            dp = p1 - b.y;
        }
    };
    float dr0, dp0, dr1 = 0.f, dp1 = 0.f;
    diff(ux, uy, uz, dr0, dp0);
    if (D == 3) diff(vx, vy, vz, dr1, dp1);
    const float nr = sqrtf(dr0 * dr0 + dr1 * dr1), npp = sqrtf(dp0 * dp0 + dp1 * dp1);
    const float dot = dr0 * dp0 + dr1 * dp1;
    // interface identification (Sec. IV.B): 0 = 1-2, 1 = 1-3, 2 = 2-3
    int pair;
    if (nr < 0.01f * (p.rho_l - p.rho_g) * p.inv_chi * npp) pair = 2;
    else if (r1 > 0.5f * p.rho_l && p1 < -0.95f * p.chi) pair = 1;
    else if (r1 > 0.5f * p.rho_l && p1 > 0.95f * p.chi) pair = 0;
    else if (dot < 0.f) pair = 1;
    else pair = 0;
    const float dc0 = pair == 2 ? dp0 : dr0, dc1 = pair == 2 ? dp1 : dr1;
    const float nc = pair == 2 ? npp : nr;
    const float cot = pair == 0 ? p.cot[0] : (pair == 1 ? p.cot[1] : p.cot[2]);
    if (!(nc > 1e-12f)) { gr = r1; gp = p1; return; }
    const float tx = dc0 / nc, ty = D == 3 ? dc1 / nc : 0.f;
    if (p.wetting == TLB_WET_GEOM_EXTRAP) {
        // Eqs. geomamgle, geomding; the second field follows the same interface
        const float sr = dr0 * tx + (D == 3 ? dr1 * ty : 0.f);
        const float sp = dp0 * tx + (D == 3 ? dp1 * ty : 0.f);
        gr = r1 + cot * sr;
        gp = p1 + cot * sp;
        return;
    }
    // geometric interpolation: sample at cot(theta) t_hat in the first fluid layer
    auto samp = [&](int k1, int k2, float &vr, float &vp) {
        float2 a;
        if (acc.get(yx + k1 * ux + k2 * vx, yy + k1 * uy + k2 * vy, yz + k1 * uz + k2 * vz, a)) {
            vr = a.x;
            vp = a.y;
        } else {
            vr = r1;
            vp = p1;
        }
    };
    if (D == 2) {
        const float l = cot * tx;
        const int l0 = (int)floorf(l), l1 = l0 + 1;
        float v0r, v0p, v1r, v1p;
        samp(l0, 0, v0r, v0p);
        samp(l1, 0, v1r, v1p);
        const float t = l - (float)l0;           // linear interpolation on [l0, l1] (Eq. interp2D)
        gr = v0r + t * (v1r - v0r);
        gp = v0p + t * (v1p - v0p);
        return;
    }
    const float lx = cot * tx, ly = cot * ty;
    if (sqrtf(lx * lx + ly * ly) < 1e-12f) { gr = r1; gp = p1; return; }
    const int X0 = (int)floorf(lx), Y0 = (int)floorf(ly);
    // of the four corners k = 0..3 at (X0 + (k & 1), Y0 + (k >> 1)) of the unit
    // cell around (lx, ly), drop the one nearest to the origin (first of
    // (0,0),(1,0),(0,1),(1,1) on ties) (Eq. interp3D); keep the other three in order
    int drop = 0, best = X0 * X0 + Y0 * Y0;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const int cx = X0 + (k & 1), cy = Y0 + (k >> 1);
        const int d2 = cx * cx + cy * cy;
        if (d2 < best) { best = d2; drop = k; }
    }
    const int ka = drop == 0 ? 1 : 0, kb = drop <= 1 ? 2 : 1, kc = drop <= 2 ? 3 : 2;
    const int ax = X0 + (ka & 1), ay = Y0 + (ka >> 1), bx = X0 + (kb & 1), by = Y0 + (kb >> 1);
    const int cxx = X0 + (kc & 1), cyy = Y0 + (kc >> 1);
    float v0r, v0p, v1r, v1p, v2r, v2p;
    samp(ax, ay, v0r, v0p);
    samp(bx, by, v1r, v1p);
    samp(cxx, cyy, v2r, v2p);
    // barycentric coordinates of (lx, ly) in the triangle
    const float e1x = (float)(bx - ax), e1y = (float)(by - ay), e2x = (float)(cxx - ax), e2y = (float)(cyy - ay);
    const float det = e1x * e2y - e2x * e1y;
    const float px = lx - (float)ax, py = ly - (float)ay;
    const float b1 = (px * e2y - e2x * py) / det, b2 = (e1x * py - px * e1y) / det;
    gr = v0r + b1 * (v1r - v0r) + b2 * (v2r - v0r);
    gp = v0p + b1 * (v1p - v0p) + b2 * (v2p - v0p);
}

}  // namespace tlb
