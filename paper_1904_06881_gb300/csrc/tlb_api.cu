// tlb_api.cu -- host side of the C ABI declared in include/tlb.h: parameter
// derivation (Carnahan-Starling coexistence, Sec. II.A), mask preprocessing
// (ghost layer, wall flags, Sec. IV), buffers, kernel launches, batched
// stepping and the request server.
#include <cuda.h>            // CUtensorMap and its enums; the encoder is looked up at run time
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

// NVTX range for the duration of a scope: host-side API calls show up by name
// in Nsight Systems timelines (a few nanoseconds when no tool is attached)
namespace {
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace
#include <string>
#include <vector>

#include "../../include/tlb.h"
#include "tlb_device.cuh"
#include "tlb_internal.h"

using namespace tlb;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_errmsg;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_errmsg = buf;
    return code;
}

#define CUDA_TRY(call)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(TLB_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

extern "C" const char *tlb_strerror(int code)
{
    switch (code) {
    case TLB_OK: return "ok";
    case TLB_E_INVAL: return "invalid argument";
    case TLB_E_NOMEM: return "out of memory";
    case TLB_E_CUDA: return "CUDA error";
    case TLB_E_UNSUPPORTED: return "unsupported";
    case TLB_E_UNCALIBRATED: return "force wetting: no kappa^w and no calibration for the angles";
    case TLB_E_DIVERGED: return "non-positive density or population";
    case TLB_E_TIMEOUT: return "device wait timed out";
    case TLB_E_BUSY: return "busy";
    case TLB_E_BOUNDS: return "index outside its array (bounds-checked build)";
    case TLB_E_NOTFOUND: return "unknown ticket";
    default: return "unknown error";
    }
}

extern "C" const char *tlb_last_error_message(void) { return g_errmsg.c_str(); }

extern "C" int tlb_version(int *major, int *minor, int *sm)
{
    if (major) *major = 1;
    if (minor) *minor = 0;
    if (sm) *sm = 103;
    return TLB_OK;
}

// ---------------------------------------------------------------------------
// allocator hook
// ---------------------------------------------------------------------------
static void *(*g_alloc)(size_t, void *) = nullptr;
static void (*g_free)(void *, void *) = nullptr;
static void *g_alloc_user = nullptr;

extern "C" int tlb_set_allocator(void *(*alloc)(size_t, void *), void (*free_)(void *, void *), void *user)
{
    if ((alloc == nullptr) != (free_ == nullptr)) return fail(TLB_E_INVAL, "allocator and free must both be set");
    g_alloc = alloc;
    g_free = free_;
    g_alloc_user = user;
    return TLB_OK;
}

struct Block {
    void *ptr;
    bool hooked;
    void *user;
    void (*fr)(void *, void *);
};

static int dev_alloc(std::vector<Block> &owned, void **out, size_t bytes, size_t *counter)
{
    void *p = nullptr;
    bytes = std::max<size_t>(bytes, 256);
    if (g_alloc) {
        p = g_alloc(bytes, g_alloc_user);
        if (!p) return fail(TLB_E_NOMEM, "allocator returned NULL for %zu bytes", bytes);
        owned.push_back({p, true, g_alloc_user, g_free});
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return fail(TLB_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        owned.push_back({p, false, nullptr, nullptr});
    }
    if (counter) *counter += bytes;
    *out = p;
    return TLB_OK;
}

static void dev_free_all(std::vector<Block> &owned)
{
    for (auto &b : owned) {
        if (b.hooked) b.fr(b.ptr, b.user);
        else cudaFree(b.ptr);
    }
    owned.clear();
}

// ---------------------------------------------------------------------------
// Carnahan-Starling EOS (Sec. II.A), host FP64.  Coexistence from the
// textbook CS pressure and chemical potential; C and Psi0 from the printed
// Psi_eos and its derivative.
// ---------------------------------------------------------------------------
namespace {
// Equations of state on the host (FP64): Carnahan-Starling (Eq. PsiEOS,
// the paper's), van der Waals and Peng-Robinson (named in Sec. II.A as EOS
// the model hosts).  p and mu are the textbook pressure and chemical
// potential; psi_printed/dpsi_printed are Psi_eos and its derivative with
// the constant C (for CS the printed formulas).  PR: attraction a A(T),
// A = (1 + k (1 - sqrt(T/T_c)))^2, k = 0.37464 + 1.54226 omega - 0.26992
// omega^2, T_c = (0.07780 / 0.45724) a / (b R).
struct CS {
    double a, b, R, T;
    int kind = TLB_EOS_CS;
    double omega = 0.344;
    double aA() const
    {
        double k = 0.37464 + 1.54226 * omega - 0.26992 * omega * omega;
        double s = 1.0 + k * (1.0 - std::sqrt(T / ((0.07780 / 0.45724) * a / (b * R))));
        return a * s * s;
    }
    double top() const { return kind == TLB_EOS_CS ? 4.0 / b : 1.0 / b; }
    double p(double r) const
    {
        if (kind == TLB_EOS_VDW) return r * R * T / (1 - b * r) - a * r * r;
        if (kind == TLB_EOS_PR) return r * R * T / (1 - b * r) - aA() * r * r / (1 + 2 * b * r - b * b * r * r);
        double e = b * r / 4.0;
        return r * R * T * (1 + e + e * e - e * e * e) / std::pow(1 - e, 3) - a * r * r;
    }
    double mu(double r) const
    {
        if (kind != TLB_EOS_CS) return dpsi_printed(r, 0.0);
        double e = b * r / 4.0;
        return R * T * (std::log(r) + (8 * e - 9 * e * e + 3 * e * e * e) / std::pow(1 - e, 3)) - 2 * a * r;
    }
    double dp(double r) const
    {
        if (kind == TLB_EOS_VDW) return R * T / ((1 - b * r) * (1 - b * r)) - 2 * a * r;
        if (kind == TLB_EOS_PR) {
            double den = 1 + 2 * b * r - b * b * r * r;
            return R * T / ((1 - b * r) * (1 - b * r)) -
                   aA() * (2 * r * den - r * r * (2 * b - 2 * b * b * r)) / (den * den);
        }
        double e = b * r / 4.0, om = 1 - e;
        double Z = (1 + e + e * e - e * e * e) / (om * om * om);
        double dZ = ((1 + 2 * e - 3 * e * e) * om + 3 * (1 + e + e * e - e * e * e)) / (om * om * om * om);
        return R * T * (Z + e * dZ) - 2 * a * r;
    }
    double psi_printed(double r, double C) const
    {
        if (kind == TLB_EOS_VDW) return r * (C - a * r + R * T * std::log(r / (1 - b * r)));
        if (kind == TLB_EOS_PR) {
            const double s2 = std::sqrt(2.0);
            return r * (C + R * T * std::log(r / (1 - b * r)) -
                        aA() / (2 * s2 * b) * std::log((b * r + s2 - 1) / (s2 + 1 - b * r)));
        }
        double br = b * r;
        return r * (C - a * r - 8 * R * T * (br - 6) / ((br - 4) * (br - 4)) + R * T * std::log(r));
    }
    double dpsi_printed(double r, double C) const
    {
        if (kind == TLB_EOS_VDW) return C - 2 * a * r + R * T * std::log(r / (1 - b * r)) + R * T / (1 - b * r);
        if (kind == TLB_EOS_PR) {
            const double s2 = std::sqrt(2.0), br = b * r, A = aA();
            return C + R * T * std::log(r / (1 - br)) + R * T / (1 - br) -
                   A / (2 * s2 * b) * std::log((br + s2 - 1) / (s2 + 1 - br)) - A * r / (1 + 2 * br - br * br);
        }
        double br = b * r, q = br - 4;
        return C - 2 * a * r + R * T * (1 + std::log(r)) + 16 * R * T * (br - 12) / (q * q * q);
    }
    // unstable interval [s1, s2] where dp/drho < 0
    bool spinodal(double &s1, double &s2) const
    {
        const int M = 6000;
        double tp = top();
        int k1 = -1, k2 = -1;
        for (int k = 1; k < M; ++k)
            if (dp(tp * k / M) < 0) {
                if (k1 < 0) k1 = k;
                k2 = k;
            }
        if (k1 < 0) return false;
        double lo = tp * (k1 - 1) / M, hi = tp * k1 / M;
        for (int it = 0; it < 120; ++it) {
            double m = 0.5 * (lo + hi);
            (dp(m) < 0 ? hi : lo) = m;
        }
        s1 = hi;
        lo = tp * k2 / M;
        hi = tp * (k2 + 1) / M;
        for (int it = 0; it < 120; ++it) {
            double m = 0.5 * (lo + hi);
            (dp(m) < 0 ? lo : hi) = m;
        }
        s2 = lo;
        return true;
    }
    // coexistence by a search over ln(rho_g): the liquid root of p(rho_l) = p(rho_g)
    // beyond the spinodal, then mu(rho_l) = mu(rho_g)
    bool coexist(double &rg, double &rl) const
    {
        double s1, s2;
        if (!spinodal(s1, s2)) return false;
        double pmin = p(s2), pmax = p(s1);
        auto liquid_for = [&](double pg) {
            double lo = s2, hi = top() * (1 - 1e-14);
            for (int it = 0; it < 200; ++it) {
                double m = 0.5 * (lo + hi);
                (p(m) < pg ? lo : hi) = m;
            }
            return 0.5 * (lo + hi);
        };
        // admissible gas densities: p(rho_g) in (max(pmin, 0), pmax)
        double lgl = std::log(1e-300), lgh = std::log(s1);
        // lower end: the smallest rho_g with p(rho_g) > pmin
        if (pmin > 0) {
            double lo = lgl, hi = lgh;
            for (int it = 0; it < 200; ++it) {
                double m = 0.5 * (lo + hi);
                (p(std::exp(m)) < pmin ? lo : hi) = m;
            }
            lgl = hi;
        }
        (void)pmax;
        auto G = [&](double lg) {
            double r = std::exp(lg);
            return mu(liquid_for(p(r))) - mu(r);
        };
        double glo = G(lgl);
        for (int it = 0; it < 200; ++it) {
            double m = 0.5 * (lgl + lgh);
            double gm = G(m);
            if ((gm < 0) == (glo < 0)) { lgl = m; glo = gm; } else lgh = m;
            if (lgh - lgl < 1e-15) break;
        }
        rg = std::exp(0.5 * (lgl + lgh));
        rl = liquid_for(p(rg));
        return true;
    }
};

double critical_T(double a, double b, double R, int kind, double omega)
{
    double lo = 0.01 * a / (b * R), hi = a / (b * R);
    for (int it = 0; it < 80; ++it) {
        double m = 0.5 * (lo + hi);
        double s1, s2;
        CS e{a, b, R, m, kind, omega};
        (e.spinodal(s1, s2) ? lo : hi) = m;
    }
    return 0.5 * (lo + hi);
}
}  // namespace

extern "C" int tlb_params_default(tlb_params *p)
{
    if (!p) return fail(TLB_E_INVAL, "null params");
    std::memset(p, 0, sizeof(*p));
    p->lattice = TLB_D2Q9;
    p->nx = p->ny = 64;
    p->nz = 1;
    p->lambda[0] = 0.6; p->lambda[1] = 1.0; p->lambda[2] = 1.0;
    p->kappa[0] = 0.01; p->kappa[1] = 1.0; p->kappa[2] = 1.0;
    p->chi = 5.0;
    p->a = 0.037; p->b = 0.2; p->R = 1.0;
    p->rho_l = 6.143914427184784;
    p->rho_g = 0.43446462473239633;
    p->beta = 0.5;
    p->tau_g = 1.0;
    p->Gamma = 1.0;
    p->wetting = TLB_WET_FORCE;
    p->theta_deg[0] = p->theta_deg[1] = p->theta_deg[2] = 90.0;
    p->eos = TLB_EOS_CS;
    p->omega = 0.344;
    return TLB_OK;
}

static int derive_uncached(const tlb_params &p, tlb_derived &d);

// The coexistence solve takes tens of milliseconds; contexts created with the
// same EOS constants and densities (every request of a served mix) reuse it.
static int derive(const tlb_params &p, tlb_derived &d)
{
    struct Key {
        double a, b, R, rho_l, rho_g, k0, k1, k2, chi, omega, eos;
        bool operator==(const Key &o) const { return std::memcmp(this, &o, sizeof(Key)) == 0; }
    };
    static std::mutex mu;
    static std::vector<std::pair<Key, tlb_derived>> cache;
    Key k = {p.a, p.b, p.R, p.rho_l, p.rho_g, p.kappa[0], p.kappa[1], p.kappa[2], p.chi, p.omega, (double)p.eos};
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &e : cache)
            if (e.first == k) {
                d = e.second;
                return TLB_OK;
            }
    }
    int rc = derive_uncached(p, d);
    if (rc == TLB_OK) {
        std::lock_guard<std::mutex> lk(mu);
        if (cache.size() >= 16) cache.erase(cache.begin());
        cache.push_back({k, d});
    }
    return rc;
}

static int derive_uncached(const tlb_params &p, tlb_derived &d)
{
    if (!(p.rho_l > p.rho_g && p.rho_g > 0)) return fail(TLB_E_INVAL, "need rho_l > rho_g > 0");
    if (!(p.a > 0 && p.b > 0 && p.R > 0)) return fail(TLB_E_INVAL, "EOS constants must be positive");
    double Tc = critical_T(p.a, p.b, p.R, p.eos, p.omega);
    double ratio = p.rho_l / p.rho_g;
    // the density ratio fixes T; bisection on T/T_c
    double lo = 0.02, hi = 0.9999, rg = 0, rl = 0;
    for (int it = 0; it < 64; ++it) {
        double m = 0.5 * (lo + hi);
        CS e{p.a, p.b, p.R, m * Tc, p.eos, p.omega};
        if (!e.coexist(rg, rl)) { hi = m; continue; }
        (rl / rg > ratio ? lo : hi) = m;
    }
    double T = 0.5 * (lo + hi) * Tc;
    CS e0{p.a, p.b, p.R, T, p.eos, p.omega};
    if (!e0.coexist(rg, rl)) return fail(TLB_E_INVAL, "no coexistence for density ratio %g", ratio);
    // scaling a, b by s keeps T_c and the ratio and divides the densities by s
    double s = rl / p.rho_l;
    CS e{p.a * s, p.b * s, p.R, T, p.eos, p.omega};
    if (!e.coexist(rg, rl)) return fail(TLB_E_INVAL, "no coexistence after rescaling");
    d.T = T;
    d.a = e.a;
    d.b = e.b;
    d.R = p.R;
    d.Tc = Tc;
    d.rho_g = rg;
    d.rho_l = rl;
    d.C = -e.dpsi_printed(rl, 0.0);
    d.Psi0 = e.psi_printed(rl, d.C);
    d.aA = p.eos == TLB_EOS_PR ? e.aA() : e.a;
    double drho = rl - rg;
    d.kappa_rr = p.kappa[0] + (p.kappa[1] + p.kappa[2]) / (4 * drho * drho);
    d.kappa_pp = (p.kappa[1] + p.kappa[2]) / (4 * p.chi * p.chi);
    d.kappa_rp = (p.kappa[1] - p.kappa[2]) / (4 * p.chi * drho);
    return TLB_OK;
}

static DevParams make_dev(const tlb_params &p, const tlb_derived &d)
{
    DevParams q;
    std::memset(&q, 0, sizeof(q));
    q.nx = p.nx;
    q.ny = p.ny;
    q.nz = p.nz;
    q.N = (long long)p.nx * p.ny * p.nz;
    q.lam1 = (float)p.lambda[0];
    q.lam2 = (float)p.lambda[1];
    q.lam3 = (float)p.lambda[2];
    q.chi = (float)p.chi;
    q.inv_chi = (float)(1.0 / p.chi);
    q.a = (float)d.a;
    q.b = (float)d.b;
    q.RT = (float)(d.R * d.T);
    q.C = (float)d.C;
    q.Psi0 = (float)d.Psi0;
    q.rho_l = (float)d.rho_l;
    q.rho_g = (float)d.rho_g;
    q.inv_drho = (float)(1.0 / (d.rho_l - d.rho_g));
    q.inv_rgl = (float)(1.0 / (d.rho_g - d.rho_l));
    q.krr = (float)d.kappa_rr;
    q.kpp = (float)d.kappa_pp;
    q.krp = (float)d.kappa_rp;
    q.beta = (float)p.beta;
    q.inv_tau_g = (float)(1.0 / p.tau_g);
    q.Gamma = (float)p.Gamma;
    q.wetting = p.wetting;
    for (int k = 0; k < 3; ++k) q.cot[k] = (float)(1.0 / std::tan(p.theta_deg[k] * M_PI / 180.0));
    q.kw_rho = (float)p.kw_rho;
    q.kw_phi = (float)p.kw_phi;
    q.g_fp16 = p.g_fp16;
    q.g_scale = p.g_fp16 ? 16.0f : 1.0f;        // moving g populations are O(0.1) or smaller
    q.g_unscale = p.g_fp16 ? 1.0f / 16.0f : 1.0f;
    q.eos = p.eos;
    q.aA = (float)d.aA;
    q.nu_on = (p.nu[0] > 0 || p.nu[1] > 0 || p.nu[2] > 0) ? 1 : 0;
    for (int k = 0; k < 3; ++k) q.nu[k] = (float)p.nu[k];
    return q;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct tlb_ctx {
    tlb_params p;
    tlb_derived d;
    DevParams dp;
    DevState s;
    int D, Q;
    long long N;
    cudaStream_t stream = nullptr;
    std::vector<Block> owned;
    size_t bytes = 0;
    std::vector<uint8_t> type_host;
    std::vector<int> ghost_host;
    int *ghosts_dev = nullptr;
    size_t ghosts_cap = 0;
    double *diag_part = nullptr, *diag_out = nullptr;
    int diag_nb = 0;
    long long steps = 0;
    long long launches = 0;
    int sticky = TLB_OK;
    // the lattice as a batch of one: entries for both buffer parities, tile table
    CUtensorMap *tmaps = nullptr;     // D3Q27: per parity, tensor maps of f_in and g_in (null if unused)
    BatchEntry *self_entries = nullptr;
    int4 *self_tiles = nullptr;
    int nself_tiles = 0;
    // one CUDA graph per buffer parity holding the launches of a step (D3Q27)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
};

static void drop_graphs(tlb_ctx *c)
{
    for (int k = 0; k < 2; ++k)
        if (c->gexec[k]) {
            cudaGraphExecDestroy(c->gexec[k]);
            c->gexec[k] = nullptr;
        }
}

static int Qof(int lattice) { return lattice == TLB_D3Q27 ? 27 : 9; }

// bytes of one copy of the g populations: FP32 [Q][N], or g_0 in FP32 plus the
// moving populations in FP16
static size_t g_bytes(int lattice, size_t N, int fp16)
{
    size_t Q = (size_t)Qof(lattice);
    return fp16 ? N * 4 + (Q - 1) * N * 2 : Q * N * 4;
}
static int Dof(int lattice) { return lattice == TLB_D3Q27 ? 3 : 2; }

#define DISPATCH(ctx, call)                       \
    do {                                          \
        if ((ctx)->D == 2) Launch<2>::call;       \
        else Launch<3>::call;                     \
    } while (0)

static int check_launch(tlb_ctx *c, int nlaunch)
{
    c->launches += nlaunch;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TLB_E_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    return TLB_OK;
}

static int validate(const tlb_params &p)
{
    if (p.lattice != TLB_D2Q9 && p.lattice != TLB_D3Q27) return fail(TLB_E_INVAL, "lattice must be D2Q9 or D3Q27");
    if (p.nx < 3 || p.ny < 3 || p.nz < 1) return fail(TLB_E_INVAL, "lattice too small (%d x %d x %d)", p.nx, p.ny, p.nz);
    if (p.lattice == TLB_D2Q9 && p.nz != 1) return fail(TLB_E_INVAL, "D2Q9 needs nz = 1");
    if (p.lattice == TLB_D3Q27 && p.nz < 3) return fail(TLB_E_INVAL, "D3Q27 needs nz >= 3");
    if ((long long)p.nx * p.ny * p.nz > (1LL << 31) - 1) return fail(TLB_E_INVAL, "more than 2^31-1 nodes");
    if (!(p.beta > 0 && p.beta <= 1)) return fail(TLB_E_INVAL, "beta must lie in (0, 1]");
    if (!(p.tau_g >= 0.5)) return fail(TLB_E_INVAL, "tau_g must be >= 0.5");
    if (!(p.chi > 0)) return fail(TLB_E_INVAL, "chi must be positive");
    if (p.wetting < 0 || p.wetting > 2) return fail(TLB_E_INVAL, "unknown wetting scheme");
    if (p.eos < TLB_EOS_CS || p.eos > TLB_EOS_PR) return fail(TLB_E_INVAL, "unknown equation of state");
    for (int k = 0; k < 3; ++k)
        if (!(p.nu[k] >= 0)) return fail(TLB_E_INVAL, "viscosities must be >= 0");
    for (int k = 0; k < 3; ++k) {
        double t = p.theta_deg[k];
        if (p.wetting != TLB_WET_FORCE && !(t >= 20.0 && t <= 160.0))
            return fail(TLB_E_UNSUPPORTED, "geometric wetting supports angles in [20, 160] deg (got %g)", t);
        if (!(t > 0 && t < 180)) return fail(TLB_E_INVAL, "angle out of (0, 180)");
    }
    return TLB_OK;
}

#define ALLOC_LATE(field, nbytes)                                        \
    do {                                                                 \
        void *p_ = nullptr;                                              \
        rc = dev_alloc(c->owned, &p_, (nbytes), &c->bytes);              \
        if (rc) { dev_free_all(c->owned); delete c; return rc; }         \
        field = (decltype(field))p_;                                     \
    } while (0)

// cuTensorMapEncodeTiled from the driver, looked up once (the library does not
// link against libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return fn;
}

// D3Q27: tensor maps of both parities' input populations, for the step
// kernel's TMA copies of a tile's own nodes (a box of TX x TY x TZ nodes and
// all directions; the copy lands in the layout [direction][z][y][x] of the
// staging area).  Per parity: f, then FP32 g, or the FP32 rest channel of g and
// its FP16 moving channels.  Every global stride must be a multiple of 16
// bytes: nx % 4 == 0 (FP32 arrays), nx % 8 == 0 (FP16 channels).  Returns false
// when the lattice does not qualify or the driver offers no encoder; the kernel
// then copies with per-thread cp.async.
static bool encode_tensor_maps(const tlb_ctx *c, CUtensorMap maps[6])
{
    if (c->D != 3) return false;
    const bool half = c->p.g_fp16 != 0;
    const cuuint64_t nx = c->p.nx, ny = c->p.ny, nz = c->p.nz, N = (cuuint64_t)c->N;
    if (nx % (half ? 8 : 4) != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint32_t box[4] = {(cuuint32_t)Launch<3>::tile_dims(0), (cuuint32_t)Launch<3>::tile_dims(1),
                               (cuuint32_t)Launch<3>::tile_dims(2), 0};
    auto tiled = [&](CUtensorMap *m, CUtensorMapDataType dt, cuuint64_t esz, const void *base, cuuint32_t depth) {
        if ((uintptr_t)base & 15) return false;
        const cuuint32_t rank = depth > 1 ? 4 : 3;
        const cuuint64_t dims[4] = {nx, ny, nz, depth};
        const cuuint64_t strides[3] = {nx * esz, nx * ny * esz, N * esz};
        const cuuint32_t b[4] = {box[0], box[1], box[2], depth};
        const cuuint32_t one[4] = {1, 1, 1, 1};
        return enc(m, dt, rank, const_cast<void *>(base), dims, strides, b, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    memset(maps, 0, 6 * sizeof(CUtensorMap));
    const cuuint32_t Q = (cuuint32_t)c->Q;
    for (int par = 0; par < 2; ++par) {
        CUtensorMap *m = maps + 3 * par;
        if (!tiled(&m[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->s.f[par], Q)) return false;
        if (!half) {
            if (!tiled(&m[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->s.g[par], Q)) return false;
        } else {
            if (!tiled(&m[1], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, c->s.g[par], 1)) return false;
            if (!tiled(&m[2], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (const char *)c->s.g[par] + 4 * N, Q - 1))
                return false;
        }
    }
    return true;
}

// the entry's tensor-map pointers for input buffer `cur` (all null without maps)
static void entry_maps(const tlb_ctx *c, int cur, BatchEntry &e)
{
    for (int k = 0; k < 3; ++k) e.tm[k] = c->tmaps ? (const void *)(c->tmaps + 3 * cur + k) : nullptr;
}

// ---------------------------------------------------------------------------
// Force-wetting calibration (no counterpart in the paper, whose wetting force
// of Eq. forceBC takes strengths, not angles): registered tables of measured
// (kappa^w, theta) pairs of a liquid drop on a wall, per lattice and
// thermodynamic parameter set.
// ---------------------------------------------------------------------------
namespace {
struct ForceTable {
    tlb_params key;
    std::vector<double> kw, th;      // th strictly decreasing in kw
};
std::mutex g_cal_mutex;
std::vector<ForceTable> g_cal;

bool same_set(const tlb_params &a, const tlb_params &b)
{
    auto eq = [](double x, double y) { return std::fabs(x - y) <= 1e-9 * std::max(1.0, std::fabs(x)); };
    if (a.lattice != b.lattice) return false;
    for (int k = 0; k < 3; ++k)
        if (!eq(a.lambda[k], b.lambda[k]) || !eq(a.kappa[k], b.kappa[k])) return false;
    return eq(a.chi, b.chi) && eq(a.rho_l, b.rho_l) && eq(a.rho_g, b.rho_g) && eq(a.a, b.a) && eq(a.b, b.b) &&
           eq(a.R, b.R);
}

// strength for angle th by linear interpolation in the table; false outside it
bool table_kw(const ForceTable &t, double th, double &kw)
{
    const size_t n = t.th.size();
    if (!(th <= t.th.front() && th >= t.th.back())) return false;
    for (size_t i = 0; i + 1 < n; ++i)
        if (th <= t.th[i] && th >= t.th[i + 1]) {
            const double s = (t.th[i] - th) / (t.th[i] - t.th[i + 1]);
            kw = t.kw[i] + s * (t.kw[i + 1] - t.kw[i]);
            return true;
        }
    return false;
}

// Force wetting with angles and no strengths: the liquid-gas angles theta_21
// (liquid 2) and theta_31 (liquid 3) map to the strengths s2, s3 of the two
// liquids, kappa_rho^w = (s2 + s3)/2, kappa_phi^w = (s2 - s3)/2 (rho^rel = 1,
// phi^rel = +-1 in Eq. forceBC).  theta_23 is not an input of this scheme.
int apply_force_calibration(tlb_params &p)
{
    if (p.wetting != TLB_WET_FORCE || p.kw_rho != 0.0 || p.kw_phi != 0.0) return TLB_OK;
    if (p.theta_deg[0] == 90.0 && p.theta_deg[1] == 90.0) return TLB_OK;
    std::lock_guard<std::mutex> lk(g_cal_mutex);
    for (const ForceTable &t : g_cal) {
        if (!same_set(t.key, p)) continue;
        double s2 = 0.0, s3 = 0.0;
        if (!table_kw(t, p.theta_deg[0], s2) || !table_kw(t, p.theta_deg[1], s3))
            return fail(TLB_E_UNCALIBRATED, "force wetting: angles (%g, %g) outside the calibrated range [%g, %g] deg",
                        p.theta_deg[0], p.theta_deg[1], t.th.back(), t.th.front());
        p.kw_rho = 0.5 * (s2 + s3);
        p.kw_phi = 0.5 * (s2 - s3);
        return TLB_OK;
    }
    return fail(TLB_E_UNCALIBRATED, "force wetting: no calibration table for this lattice and parameter set "
                                    "(pass kw_rho, kw_phi, or register one with tlb_set_force_calibration)");
}
}  // namespace

extern "C" int tlb_set_force_calibration(const tlb_params *p, const double *kappa_w, const double *theta_deg, int n)
{
    if (!p || !kappa_w || !theta_deg) return fail(TLB_E_INVAL, "null argument");
    if (n < 2) return fail(TLB_E_INVAL, "a calibration table needs at least two points");
    ForceTable t;
    t.key = *p;
    for (int i = 0; i < n; ++i) {
        if (!std::isfinite(kappa_w[i]) || !std::isfinite(theta_deg[i]))
            return fail(TLB_E_INVAL, "non-finite calibration point %d", i);
        if (i > 0 && !(kappa_w[i] > kappa_w[i - 1] && theta_deg[i] < theta_deg[i - 1]))
            return fail(TLB_E_INVAL, "calibration points must increase in kappa^w and decrease in theta (point %d)", i);
        t.kw.push_back(kappa_w[i]);
        t.th.push_back(theta_deg[i]);
    }
    std::lock_guard<std::mutex> lk(g_cal_mutex);
    for (ForceTable &u : g_cal)
        if (same_set(u.key, *p)) {
            u = t;
            return TLB_OK;
        }
    g_cal.push_back(t);
    return TLB_OK;
}

extern "C" int tlb_derive(const tlb_params *p, tlb_derived *out)
{
    if (!p || !out) return fail(TLB_E_INVAL, "null argument");
    int rc = validate(*p);
    if (rc) return rc;
    return derive(*p, *out);
}

extern "C" int tlb_create_ex(const tlb_params *pin, tlb_ctx **out)
{
    if (!pin || !out) return fail(TLB_E_INVAL, "null argument");
    *out = nullptr;
    tlb_params pc = *pin;
    int rc = apply_force_calibration(pc);
    if (rc) return rc;
    pin = &pc;
    rc = validate(*pin);
    if (rc) return rc;
    tlb_ctx *c = new tlb_ctx();
    c->p = *pin;
    rc = derive(c->p, c->d);
    if (rc) { delete c; return rc; }
    c->dp = make_dev(c->p, c->d);
    c->D = Dof(c->p.lattice);
    c->Q = Qof(c->p.lattice);
    c->N = c->dp.N;
    size_t N = (size_t)c->N, Q = (size_t)c->Q;
    size_t gb = g_bytes(c->p.lattice, N, c->p.g_fp16);
    void *ptr;
#define ALLOC(field, nbytes)                                             \
    do {                                                                 \
        rc = dev_alloc(c->owned, &ptr, (nbytes), &c->bytes);             \
        if (rc) { dev_free_all(c->owned); delete c; return rc; }         \
        field = (decltype(field))ptr;                                    \
    } while (0)
    ALLOC(c->s.f[0], Q * N * 4);
    ALLOC(c->s.f[1], Q * N * 4);
    ALLOC(c->s.g[0], gb);
    ALLOC(c->s.g[1], gb);
    ALLOC(c->s.rho, N * 4);
    ALLOC(c->s.phi, N * 4);
    ALLOC(c->s.type, N);
    ALLOC(c->s.status, 256);
    c->diag_nb = c->D == 2 ? Launch<2>::diag_blocks(c->dp) : Launch<3>::diag_blocks(c->dp);
    ALLOC(c->diag_part, (size_t)c->diag_nb * 6 * 8);
    ALLOC(c->diag_out, 6 * 8);
#undef ALLOC
    c->s.cur = 0;
    c->s.ghosts = nullptr;
    c->s.nghost = 0;
    cudaMemsetAsync(c->s.type, 0, N, c->stream);
    cudaMemsetAsync(c->s.status, 0, 256, c->stream);
    cudaMemsetAsync(c->s.f[0], 0, Q * N * 4, c->stream);
    cudaMemsetAsync(c->s.g[0], 0, gb, c->stream);
    cudaMemsetAsync(c->s.f[1], 0, Q * N * 4, c->stream);
    cudaMemsetAsync(c->s.g[1], 0, gb, c->stream);
    cudaMemsetAsync(c->s.rho, 0, N * 4, c->stream);
    cudaMemsetAsync(c->s.phi, 0, N * 4, c->stream);
    c->type_host.assign(N, 0);
    {
        CUtensorMap maps[6];
        if (encode_tensor_maps(c, maps)) {
            ALLOC_LATE(c->tmaps, sizeof(maps));
            if ((uintptr_t)c->tmaps & 63) {
                c->tmaps = nullptr;           // a tensor map in global memory needs 64-byte alignment
            } else {
                cudaMemcpyAsync(c->tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, c->stream);
            }
        }
    }
    {
        // batch-of-one tables: entry per buffer parity, one tile per CTA
        int D = c->D;
        int TX = D == 2 ? Launch<2>::tile_dims(0) : Launch<3>::tile_dims(0);
        int TY = D == 2 ? Launch<2>::tile_dims(1) : Launch<3>::tile_dims(1);
        int TZ = D == 2 ? Launch<2>::tile_dims(2) : Launch<3>::tile_dims(2);
        std::vector<int4> tiles;
        for (int z = 0; z < c->p.nz; z += TZ)
            for (int y = 0; y < c->p.ny; y += TY)
                for (int x = 0; x < c->p.nx; x += TX) tiles.push_back(make_int4(0, x, y, z));
        BatchEntry ent[2];
        for (int par = 0; par < 2; ++par) {
            ent[par].p = c->dp;
            ent[par].f_in = c->s.f[par];
            ent[par].f_out = c->s.f[1 - par];
            ent[par].g_in = c->s.g[par];
            ent[par].g_out = c->s.g[1 - par];
            ent[par].rho = c->s.rho;
            ent[par].phi = c->s.phi;
            ent[par].type = c->s.type;
            ent[par].status = c->s.status;
            entry_maps(c, par, ent[par]);
        }
        ALLOC_LATE(c->self_entries, sizeof(ent));
        ALLOC_LATE(c->self_tiles, tiles.size() * sizeof(int4));
        c->nself_tiles = (int)tiles.size();
        cudaMemcpyAsync(c->self_entries, ent, sizeof(ent), cudaMemcpyHostToDevice, c->stream);
        cudaMemcpyAsync(c->self_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        dev_free_all(c->owned);
        delete c;
        return fail(TLB_E_CUDA, "create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return TLB_OK;
}

extern "C" int tlb_create(int lattice, int nx, int ny, int nz, const double densities[2], const double kappas[3],
                          const double viscosities[3], int wetting, const double angles_deg[3], tlb_ctx **out)
{
    if (!densities || !kappas || !viscosities || !angles_deg || !out) return fail(TLB_E_INVAL, "null argument");
    tlb_params p;
    tlb_params_default(&p);
    p.lattice = lattice;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.rho_l = densities[0];
    p.rho_g = densities[1];
    for (int k = 0; k < 3; ++k) p.kappa[k] = kappas[k];
    for (int k = 0; k < 3; ++k)
        if (!(viscosities[k] > 0)) return fail(TLB_E_INVAL, "viscosities must be positive");
    p.beta = 1.0 / (1.0 + 6.0 * viscosities[0]);   // nu = (1/beta - 1)/6
    if (!(viscosities[0] == viscosities[1] && viscosities[1] == viscosities[2]))
        for (int k = 0; k < 3; ++k) p.nu[k] = viscosities[k];   // per-component viscosity
    p.wetting = wetting;
    for (int k = 0; k < 3; ++k) p.theta_deg[k] = angles_deg[k];
    return tlb_create_ex(&p, out);      // force wetting: angles through the calibration tables
}

extern "C" void tlb_destroy(tlb_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    dev_free_all(c->owned);
    delete c;
}

extern "C" int tlb_get_params(const tlb_ctx *c, tlb_params *out)
{
    if (!c || !out) return fail(TLB_E_INVAL, "null argument");
    *out = c->p;
    return TLB_OK;
}

extern "C" int tlb_get_derived(const tlb_ctx *c, tlb_derived *out)
{
    if (!c || !out) return fail(TLB_E_INVAL, "null argument");
    *out = c->d;
    return TLB_OK;
}

extern "C" int tlb_set_stream(tlb_ctx *c, void *stream)
{
    if (!c) return fail(TLB_E_INVAL, "null context");
    c->stream = (cudaStream_t)stream;
    return TLB_OK;
}

// Node flags and ghost list of a periodic lattice from its solid mask (NULL:
// no walls): solid, ghost (solid with a fluid lattice neighbour), first layer
// (fluid with a solid lattice neighbour), wall axes, and NEAR (fluid off the
// first layer with a first-layer neighbour: where the wetting force acts).
static void node_flags(int nx, int ny, int nz, int D, const uint8_t *mask, std::vector<uint8_t> &t,
                       std::vector<int> &ghosts)
{
    auto at = [&](int x, int y, int z) -> long long {
        x = ((x % nx) + nx) % nx;
        y = ((y % ny) + ny) % ny;
        z = ((z % nz) + nz) % nz;
        return (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
    };
    auto solid = [&](long long n) { return mask != nullptr && mask[n] != 0; };
    long long N = (long long)nx * ny * nz;
    t.assign((size_t)N, 0);
    ghosts.clear();
    const int zr = D == 3 ? 1 : 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long long n = at(x, y, z);
                bool s = solid(n), touch = false;
                for (int dz = -zr; dz <= zr; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx)
                            if ((dx || dy || dz) && solid(at(x + dx, y + dy, z + dz)) != s) touch = true;
                uint8_t v = s ? TLB_SOLID : 0;
                if (s && touch) {
                    v |= TLB_GHOST;
                    ghosts.push_back((int)n);
                }
                if (!s) {
                    if (touch) v |= TLB_FIRST;
                    if (solid(at(x + 1, y, z)) || solid(at(x - 1, y, z))) v |= TLB_WALLX;
                    if (solid(at(x, y + 1, z)) || solid(at(x, y - 1, z))) v |= TLB_WALLY;
                    if (D == 3 && (solid(at(x, y, z + 1)) || solid(at(x, y, z - 1)))) v |= TLB_WALLZ;
                }
                t[n] = v;
            }
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long long n = at(x, y, z);
                if (t[n] & (TLB_SOLID | TLB_FIRST)) continue;
                bool near = false;
                for (int dz = -zr; dz <= zr; ++dz)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx)
                            if ((dx || dy || dz) && (t[at(x + dx, y + dy, z + dz)] & TLB_FIRST)) near = true;
                if (near) t[n] |= TLB_NEAR;
            }
}

extern "C" int tlb_set_solid(tlb_ctx *c, const uint8_t *mask)
{
    if (!c || !mask) return fail(TLB_E_INVAL, "null argument");
    long long N = c->N;
    std::vector<uint8_t> t;
    node_flags(c->p.nx, c->p.ny, c->p.nz, c->D, mask, t, c->ghost_host);
    c->type_host = t;
    drop_graphs(c);
    CUDA_TRY(cudaMemcpyAsync(c->s.type, t.data(), N, cudaMemcpyHostToDevice, c->stream));
    size_t ng = c->ghost_host.size();
    if (ng > c->ghosts_cap) {
        void *ptr;
        int rc = dev_alloc(c->owned, &ptr, ng * sizeof(int), &c->bytes);
        if (rc) return rc;
        c->ghosts_dev = (int *)ptr;
        c->ghosts_cap = ng;
    }
    if (ng) CUDA_TRY(cudaMemcpyAsync(c->ghosts_dev, c->ghost_host.data(), ng * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    c->s.ghosts = c->ghosts_dev;
    c->s.nghost = (int)ng;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return TLB_OK;
}

static int check_status(tlb_ctx *c)
{
    unsigned st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, c->s.status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (st & STATUS_TIMEOUT) {
        c->sticky = TLB_E_TIMEOUT;
        return fail(TLB_E_TIMEOUT, "a tile's tensor copies did not complete within one second");
    }
    if (st) {
        c->sticky = TLB_E_DIVERGED;
        return fail(TLB_E_DIVERGED, "non-positive density or population met");
    }
#ifdef TLB_BOUNDS_CHECK
    // the error words are per lattice type, not per context: a violation shows
    // at the next check of any context
    if (unsigned nb = Launch<2>::bounds_errors() | Launch<3>::bounds_errors()) {
        c->sticky = TLB_E_BOUNDS;
        return fail(TLB_E_BOUNDS, "bounds check: %u flagged node indices outside their arrays", nb);
    }
#endif
    return TLB_OK;
}

extern "C" int tlb_sync(tlb_ctx *c)
{
    if (!c) return fail(TLB_E_INVAL, "null context");
    return check_status(c);
}

static int init_from_device(tlb_ctx *c, const float *u_dev)
{
    DISPATCH(c, ghosts(c->dp, c->s, c->stream));
    AuxOut none = {};
    DISPATCH(c, step(c->dp, c->s, MODE_INIT, u_dev, none, c->stream));
    c->steps = 0;
    return check_launch(c, 2);
}

extern "C" int tlb_init_fields_device(tlb_ctx *c, const float *rho, const float *phi, const float *u)
{
    if (!c || !rho || !phi) return fail(TLB_E_INVAL, "null argument");
    size_t N = (size_t)c->N;
    CUDA_TRY(cudaMemcpyAsync(c->s.rho, rho, N * 4, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->s.phi, phi, N * 4, cudaMemcpyDeviceToDevice, c->stream));
    return init_from_device(c, u);
}

// temporary device buffer owned by one call
struct Scratch {
    void *p = nullptr;
    ~Scratch()
    {
        if (p) cudaFree(p);
    }
};

extern "C" int tlb_init_fields(tlb_ctx *c, const double *rho, const double *phi, const double *u)
{
    if (!c || !rho || !phi) return fail(TLB_E_INVAL, "null argument");
    size_t N = (size_t)c->N;
    std::vector<float> hr(N), hp(N), hu;
    for (size_t n = 0; n < N; ++n) {
        bool s = c->type_host[n] & TLB_SOLID;
        hr[n] = s ? 0.f : (float)rho[n];
        hp[n] = s ? 0.f : (float)phi[n];
        if (!s && !(rho[n] > 0)) return fail(TLB_E_INVAL, "rho must be positive at fluid node %zu", n);
    }
    Scratch su;
    if (u) {
        hu.resize((size_t)c->D * N);
        for (size_t k = 0; k < hu.size(); ++k) hu[k] = (float)u[k];
        CUDA_TRY(cudaMalloc(&su.p, hu.size() * 4));
        CUDA_TRY(cudaMemcpyAsync(su.p, hu.data(), hu.size() * 4, cudaMemcpyHostToDevice, c->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(c->s.rho, hr.data(), N * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->s.phi, hp.data(), N * 4, cudaMemcpyHostToDevice, c->stream));
    int rc = init_from_device(c, (const float *)su.p);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->sticky = TLB_OK;
    return TLB_OK;
}

// Launches of one step per lattice: D2Q9 one (the step kernel sums the
// moments it needs), D3Q27 two (moments, step).
static int launches_per_step(int D) { return D == 2 ? 1 : 2; }

// The launches of one step of a lattice, as a batch of one (the kernels
// tlb_step_batch uses, so alone and batched results are bit-identical).
// Phase 0 is the moments pass (D3Q27 only), phase 2 the step kernel.
static void issue_phase(tlb_ctx *c, int phase, cudaStream_t st)
{
    const BatchEntry *E = c->self_entries + c->s.cur;
    int fp16 = c->p.g_fp16;
    if (c->D == 2) {
        if (phase == 2) Launch<2>::step_batch(E, c->self_tiles, c->nself_tiles, fp16, st);
    } else {
        if (phase == 0) Launch<3>::moments_batch(E, c->self_tiles, c->nself_tiles, fp16, st);
        else if (phase == 2) Launch<3>::step_batch(E, c->self_tiles, c->nself_tiles, fp16, st);
    }
}

static void issue_step_on(tlb_ctx *c, cudaStream_t st)
{
    issue_phase(c, 0, st);
    issue_phase(c, 2, st);
}

// Capture the launches of a step for the current buffer parity.
static int capture_step(tlb_ctx *c)
{
    int par = c->s.cur;
    if (c->gexec[par]) return TLB_OK;
    if (!c->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    issue_step_on(c, c->cap_stream);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (e != cudaSuccess) return fail(TLB_E_CUDA, "step capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec[par], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec[par] = nullptr;
        return fail(TLB_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return TLB_OK;
}

extern "C" int tlb_step(tlb_ctx *c, int nsteps)
{
    NvtxRange range("tlb_step");
    if (!c) return fail(TLB_E_INVAL, "null context");
    if (nsteps < 0) return fail(TLB_E_INVAL, "nsteps < 0");
    const int per = launches_per_step(c->D);
    for (int k = 0; k < nsteps; ++k) {
        if (per == 1) {
            // a single launch: direct (a one-node graph costs more to launch)
            issue_step_on(c, c->stream);
        } else {
            int rc = capture_step(c);
            if (rc) return rc;
            CUDA_TRY(cudaGraphLaunch(c->gexec[c->s.cur], c->stream));
        }
        c->s.cur ^= 1;
        c->steps += 1;
        c->launches += per;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TLB_E_CUDA, "step launch: %s", cudaGetErrorString(e));
    return c->sticky;
}

extern "C" int tlb_step_phase(tlb_ctx *c, int phase)
{
    if (!c) return fail(TLB_E_INVAL, "null context");
    if (phase < 0 || phase > 2) return fail(TLB_E_INVAL, "phase must be 0, 1 or 2");
    if (phase == 1) return TLB_OK;        // the ghost layer is filled inside phase 2
    if (phase == 0 && c->D == 2) return TLB_OK;   // D2Q9 step kernels sum their moments
    issue_phase(c, phase, c->stream);
    if (phase == 2) {
        c->s.cur ^= 1;
        c->steps += 1;
    }
    return check_launch(c, 1);
}

extern "C" int tlb_get_fields_device(tlb_ctx *c, float *rho, float *phi, float *u)
{
    if (!c) return fail(TLB_E_INVAL, "null context");
    size_t N = (size_t)c->N;
    DISPATCH(c, moments(c->dp, c->s, c->stream));
    int nl = 1;
    if (u) {
        DISPATCH(c, fields(c->dp, c->s, u, c->stream));
        ++nl;
    }
    if (rho) CUDA_TRY(cudaMemcpyAsync(rho, c->s.rho, N * 4, cudaMemcpyDeviceToDevice, c->stream));
    if (phi) CUDA_TRY(cudaMemcpyAsync(phi, c->s.phi, N * 4, cudaMemcpyDeviceToDevice, c->stream));
    return check_launch(c, nl);
}

extern "C" int tlb_get_fields(tlb_ctx *c, double *rho, double *phi, double *u, double *C)
{
    if (!c) return fail(TLB_E_INVAL, "null context");
    size_t N = (size_t)c->N;
    Scratch su;
    std::vector<float> hr(N), hp(N), hu;
    DISPATCH(c, moments(c->dp, c->s, c->stream));
    int nl = 1;
    if (u) {
        CUDA_TRY(cudaMalloc(&su.p, (size_t)c->D * N * 4));
        DISPATCH(c, fields(c->dp, c->s, (float *)su.p, c->stream));
        ++nl;
        hu.resize((size_t)c->D * N);
        CUDA_TRY(cudaMemcpyAsync(hu.data(), su.p, hu.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(hr.data(), c->s.rho, N * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(hp.data(), c->s.phi, N * 4, cudaMemcpyDeviceToHost, c->stream));
    int rc = check_launch(c, nl);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    const double rl = c->d.rho_l, rg = c->d.rho_g, chi = c->p.chi;
    for (size_t n = 0; n < N; ++n) {
        bool s = c->type_host[n] & TLB_SOLID;
        double r = s ? 0.0 : hr[n], ph = s ? 0.0 : hp[n];
        if (rho) rho[n] = r;
        if (phi) phi[n] = ph;
        if (u)
            for (int a = 0; a < c->D; ++a) u[(size_t)a * N + n] = s ? 0.0 : hu[(size_t)a * N + n];
        if (C) {
            double C1 = (r - rl) / (rg - rl);
            C[n] = s ? 0.0 : C1;
            C[N + n] = s ? 0.0 : 0.5 * (1 + ph / chi - C1);
            C[2 * N + n] = s ? 0.0 : 0.5 * (1 - ph / chi - C1);
        }
    }
    return check_status(c);
}

extern "C" int tlb_diagnostics(tlb_ctx *c, double out[6])
{
    if (!c || !out) return fail(TLB_E_INVAL, "null argument");
    DISPATCH(c, moments(c->dp, c->s, c->stream));
    DISPATCH(c, diagnostics(c->dp, c->s, c->diag_part, c->diag_nb, c->diag_out, c->stream));
    int rc = check_launch(c, 3);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(out, c->diag_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return TLB_OK;
}

extern "C" int tlb_get_aux(tlb_ctx *c, int which, double *out)
{
    if (!c || !out) return fail(TLB_E_INVAL, "null argument");
    if (which < 0 || which > 13) return fail(TLB_E_INVAL, "which must be 0..13");
    size_t N = (size_t)c->N;
    Scratch sa;
    DISPATCH(c, moments(c->dp, c->s, c->stream));
    DISPATCH(c, ghosts(c->dp, c->s, c->stream));
    int nl = 2;
    const float *src = nullptr;
    if (which == 12) src = c->s.rho;
    else if (which == 13) src = c->s.phi;
    else {
        CUDA_TRY(cudaMalloc(&sa.p, N * 4));
        CUDA_TRY(cudaMemsetAsync(sa.p, 0, N * 4, c->stream));
        AuxOut a = {};
        float *dst = (float *)sa.p;
        if (which == 0) a.p0 = dst;
        else if (which == 1) a.mur = dst;
        else if (which == 2) a.mup = dst;
        else if (which <= 5) a.F[which - 3] = dst;
        else a.P[which - 6] = dst;
        DISPATCH(c, step(c->dp, c->s, MODE_AUX, nullptr, a, c->stream));
        ++nl;
        src = dst;
    }
    std::vector<float> h(N);
    CUDA_TRY(cudaMemcpyAsync(h.data(), src, N * 4, cudaMemcpyDeviceToHost, c->stream));
    int rc = check_launch(c, nl);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (size_t n = 0; n < N; ++n)
        out[n] = ((c->type_host[n] & TLB_SOLID) && which < 12) ? 0.0 : (double)h[n];
    return TLB_OK;
}

extern "C" int tlb_lattice_directions(int lattice, int *c, double *w)
{
    if (lattice != TLB_D2Q9 && lattice != TLB_D3Q27) return fail(TLB_E_INVAL, "bad lattice");
    int Q = Qof(lattice), D = Dof(lattice);
    for (int i = 0; i < Q; ++i) {
        double wi = 1.0;
        for (int a = 0; a < 3; ++a) {
            int v = (D == 2) ? (a < 2 ? cc<2>(i, a) : 0) : cc<3>(i, a);
            if (c) c[3 * i + a] = v;
            if (a < D) wi *= (v == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
        }
        if (w) w[i] = wi;
    }
    return Q;
}

static int pop_io(tlb_ctx *c, double *f, double *g, const double *fi, const double *gi, int dir)
{
    size_t QN = (size_t)c->Q * (size_t)c->N;
    Scratch s1, s2;
    CUDA_TRY(cudaMalloc(&s1.p, QN * 8));
    CUDA_TRY(cudaMalloc(&s2.p, QN * 8));
    if (dir == 1) {
        CUDA_TRY(cudaMemcpyAsync(s1.p, fi, QN * 8, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(s2.p, gi, QN * 8, cudaMemcpyHostToDevice, c->stream));
    }
    DISPATCH(c, convert_pop(c->dp, c->s, dir, (double *)s1.p, (double *)s2.p, c->stream));
    int rc = check_launch(c, 1);
    if (rc) return rc;
    if (dir == 0) {
        if (f) CUDA_TRY(cudaMemcpyAsync(f, s1.p, QN * 8, cudaMemcpyDeviceToHost, c->stream));
        if (g) CUDA_TRY(cudaMemcpyAsync(g, s2.p, QN * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return TLB_OK;
}

extern "C" int tlb_get_populations(tlb_ctx *c, double *f, double *g)
{
    if (!c) return fail(TLB_E_INVAL, "null context");
    return pop_io(c, f, g, nullptr, nullptr, 0);
}

extern "C" int tlb_set_populations(tlb_ctx *c, const double *f, const double *g)
{
    if (!c || !f || !g) return fail(TLB_E_INVAL, "null argument");
    return pop_io(c, nullptr, nullptr, f, g, 1);
}

struct SnapHeader {
    uint64_t magic, N, Q, gbytes;
    long long steps;
};

extern "C" size_t tlb_snapshot_bytes(const tlb_ctx *c)
{
    if (!c) return 0;
    size_t QN = (size_t)c->Q * (size_t)c->N;
    return sizeof(SnapHeader) + QN * 4 + g_bytes(c->p.lattice, (size_t)c->N, c->p.g_fp16);
}

extern "C" int tlb_snapshot(tlb_ctx *c, void *host, size_t bytes)
{
    if (!c || !host) return fail(TLB_E_INVAL, "null argument");
    if (bytes < tlb_snapshot_bytes(c)) return fail(TLB_E_INVAL, "snapshot buffer too small");
    size_t QN = (size_t)c->Q * (size_t)c->N, gb = g_bytes(c->p.lattice, (size_t)c->N, c->p.g_fp16);
    SnapHeader h = {0x544c4253u, (uint64_t)c->N, (uint64_t)c->Q, (uint64_t)gb, c->steps};
    std::memcpy(host, &h, sizeof(h));
    char *dst = (char *)host + sizeof(h);
    CUDA_TRY(cudaMemcpyAsync(dst, c->s.f[c->s.cur], QN * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(dst + QN * 4, c->s.g[c->s.cur], gb, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return TLB_OK;
}

extern "C" int tlb_restore(tlb_ctx *c, const void *host, size_t bytes)
{
    if (!c || !host) return fail(TLB_E_INVAL, "null argument");
    if (bytes < tlb_snapshot_bytes(c)) return fail(TLB_E_INVAL, "snapshot buffer too small");
    SnapHeader h;
    std::memcpy(&h, host, sizeof(h));
    size_t QN = (size_t)c->Q * (size_t)c->N, gb = g_bytes(c->p.lattice, (size_t)c->N, c->p.g_fp16);
    if (h.magic != 0x544c4253u || h.N != (uint64_t)c->N || h.Q != (uint64_t)c->Q || h.gbytes != gb)
        return fail(TLB_E_INVAL, "snapshot does not match this context");
    const char *src = (const char *)host + sizeof(h);
    CUDA_TRY(cudaMemcpyAsync(c->s.f[c->s.cur], src, QN * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->s.g[c->s.cur], src + QN * 4, gb, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->steps = h.steps;
    return TLB_OK;
}

extern "C" long long tlb_steps_done(const tlb_ctx *c) { return c ? c->steps : -1; }
extern "C" size_t tlb_device_bytes(const tlb_ctx *c) { return c ? c->bytes : 0; }
extern "C" long long tlb_launch_count(const tlb_ctx *c) { return c ? c->launches : -1; }

// ---------------------------------------------------------------------------
// batched stepping: one launch per phase over all lattices
// ---------------------------------------------------------------------------
struct BatchPlan {
    std::vector<tlb_ctx *> ctxs;
    std::vector<Block> owned;
    BatchEntry *entries[2] = {nullptr, nullptr};   // parity of the step
    int4 *tiles = nullptr;
    int ntiles = 0;
};

static int build_plan(tlb_ctx *const *ctxs, int n, BatchPlan &plan, cudaStream_t st)
{
    int D = ctxs[0]->D;
    std::vector<int4> tiles;
    std::vector<BatchEntry> e0(n), e1(n);
    int TX = D == 2 ? Launch<2>::tile_dims(0) : Launch<3>::tile_dims(0);
    int TY = D == 2 ? Launch<2>::tile_dims(1) : Launch<3>::tile_dims(1);
    int TZ = D == 2 ? Launch<2>::tile_dims(2) : Launch<3>::tile_dims(2);
    for (int k = 0; k < n; ++k) {
        tlb_ctx *c = ctxs[k];
        if (c->D != D) return fail(TLB_E_INVAL, "batched lattices must share the lattice type");
        if (c->p.g_fp16 != ctxs[0]->p.g_fp16) return fail(TLB_E_INVAL, "batched lattices must share the g storage");
        for (int par = 0; par < 2; ++par) {
            BatchEntry &e = par ? e1[k] : e0[k];
            int cur = (c->s.cur + par) & 1;
            e.p = c->dp;
            e.f_in = c->s.f[cur];
            e.f_out = c->s.f[1 - cur];
            e.g_in = c->s.g[cur];
            e.g_out = c->s.g[1 - cur];
            e.rho = c->s.rho;
            e.phi = c->s.phi;
            e.type = c->s.type;
            e.status = c->s.status;
            entry_maps(c, cur, e);
        }
        for (int z = 0; z < c->p.nz; z += TZ)
            for (int y = 0; y < c->p.ny; y += TY)
                for (int x = 0; x < c->p.nx; x += TX) tiles.push_back(make_int4(k, x, y, z));
    }
    void *ptr;
    int rc;
    if ((rc = dev_alloc(plan.owned, &ptr, n * sizeof(BatchEntry), nullptr))) return rc;
    plan.entries[0] = (BatchEntry *)ptr;
    if ((rc = dev_alloc(plan.owned, &ptr, n * sizeof(BatchEntry), nullptr))) return rc;
    plan.entries[1] = (BatchEntry *)ptr;
    if ((rc = dev_alloc(plan.owned, &ptr, tiles.size() * sizeof(int4), nullptr))) return rc;
    plan.tiles = (int4 *)ptr;
    CUDA_TRY(cudaMemcpyAsync(plan.entries[0], e0.data(), n * sizeof(BatchEntry), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(plan.entries[1], e1.data(), n * sizeof(BatchEntry), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(plan.tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    plan.ntiles = (int)tiles.size();
    plan.ctxs.assign(ctxs, ctxs + n);
    return TLB_OK;
}

static int run_plan(BatchPlan &plan, int nsteps, cudaStream_t st)
{
    int D = plan.ctxs[0]->D;
    for (int s = 0; s < nsteps; ++s) {
        const BatchEntry *E = plan.entries[s & 1];
        int fp16 = plan.ctxs[0]->p.g_fp16;
        if (D == 2) {
            Launch<2>::step_batch(E, plan.tiles, plan.ntiles, fp16, st);
        } else {
            Launch<3>::moments_batch(E, plan.tiles, plan.ntiles, fp16, st);
            Launch<3>::step_batch(E, plan.tiles, plan.ntiles, fp16, st);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TLB_E_CUDA, "batched launch: %s", cudaGetErrorString(e));
    const int per = launches_per_step(D);
    for (tlb_ctx *c : plan.ctxs) {
        if (nsteps & 1) c->s.cur ^= 1;
        c->steps += nsteps;
    }
    plan.ctxs[0]->launches += (long long)per * nsteps;
    return TLB_OK;
}

extern "C" int tlb_step_batch(tlb_ctx *const *ctxs, int n, int nsteps)
{
    NvtxRange range("tlb_step_batch");
    if (!ctxs || n <= 0 || nsteps < 0) return fail(TLB_E_INVAL, "bad batch arguments");
    for (int k = 0; k < n; ++k)
        if (!ctxs[k]) return fail(TLB_E_INVAL, "null context in batch");
    cudaStream_t st = ctxs[0]->stream;
    BatchPlan plan;
    int rc = build_plan(ctxs, n, plan, st);
    if (rc == TLB_OK) rc = run_plan(plan, nsteps, st);
    cudaStreamSynchronize(st);
    dev_free_all(plan.owned);
    return rc;
}

// ---------------------------------------------------------------------------
// resident batches: the tile -> lattice table built once, steps issued without
// allocation or host synchronisation, replayed from CUDA graphs of several
// steps; the launch configuration chosen by timing candidates on the batch
// ---------------------------------------------------------------------------
struct tlb_batch {
    std::vector<tlb_ctx *> ctxs;
    std::vector<int> base_cur;          // each context's buffer parity when the entries were written
    int D = 2, fp16 = 0;
    cudaStream_t st = nullptr;          // the stream of ctxs[0]
    cudaStream_t cap = nullptr;         // private stream for graph capture and tuning
    std::vector<Block> owned;
    BatchEntry *entries[2] = {nullptr, nullptr};
    int4 *tiles = nullptr;
    int ntiles = 0;
    tlb_batch_config cfg;
    // replays of cfg.graph_depth steps starting at entry parity 0 and 1
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

static void batch_drop_graphs(tlb_batch *b)
{
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) {
            cudaGraphExecDestroy(b->graph[k]);
            b->graph[k] = nullptr;
        }
}

// tile table in the configured order (written to the device table)
static std::vector<int4> batch_tile_order(const tlb_batch *b, int order)
{
    const int D = b->D;
    const int TX = D == 2 ? Launch<2>::tile_dims(0) : Launch<3>::tile_dims(0);
    const int TY = D == 2 ? Launch<2>::tile_dims(1) : Launch<3>::tile_dims(1);
    const int TZ = D == 2 ? Launch<2>::tile_dims(2) : Launch<3>::tile_dims(2);
    const int n = (int)b->ctxs.size();
    std::vector<std::vector<int4>> per(n);
    for (int k = 0; k < n; ++k) {
        const tlb_ctx *c = b->ctxs[k];
        for (int z = 0; z < c->p.nz; z += TZ)
            for (int y = 0; y < c->p.ny; y += TY)
                for (int x = 0; x < c->p.nx; x += TX) per[k].push_back(make_int4(k, x, y, z));
    }
    std::vector<int> lat(n);
    for (int k = 0; k < n; ++k) lat[k] = k;
    if (order == TLB_ORDER_LARGEST_FIRST)
        std::stable_sort(lat.begin(), lat.end(), [&](int a, int c) { return per[a].size() > per[c].size(); });
    std::vector<int4> out;
    if (order == TLB_ORDER_INTERLEAVED) {
        size_t most = 0;
        for (auto &v : per) most = std::max(most, v.size());
        for (size_t j = 0; j < most; ++j)
            for (int k = 0; k < n; ++k)
                if (j < per[k].size()) out.push_back(per[k][j]);
    } else {
        for (int k : lat) out.insert(out.end(), per[k].begin(), per[k].end());
    }
    return out;
}

// entries of both parities from the contexts' current buffers
static int batch_write_entries(tlb_batch *b)
{
    const int n = (int)b->ctxs.size();
    std::vector<BatchEntry> e[2] = {std::vector<BatchEntry>(n), std::vector<BatchEntry>(n)};
    b->base_cur.resize(n);
    for (int k = 0; k < n; ++k) {
        tlb_ctx *c = b->ctxs[k];
        b->base_cur[k] = c->s.cur;
        for (int par = 0; par < 2; ++par) {
            BatchEntry &x = e[par][k];
            int cur = (c->s.cur + par) & 1;
            x.p = c->dp;
            x.f_in = c->s.f[cur];
            x.f_out = c->s.f[1 - cur];
            x.g_in = c->s.g[cur];
            x.g_out = c->s.g[1 - cur];
            x.rho = c->s.rho;
            x.phi = c->s.phi;
            x.type = c->s.type;
            x.status = c->s.status;
            entry_maps(c, cur, x);
        }
    }
    for (int par = 0; par < 2; ++par)
        CUDA_TRY(cudaMemcpyAsync(b->entries[par], e[par].data(), n * sizeof(BatchEntry), cudaMemcpyHostToDevice,
                                 b->st));
    return TLB_OK;
}

static int batch_write_tiles(tlb_batch *b)
{
    std::vector<int4> t = batch_tile_order(b, b->cfg.tile_order);
    CUDA_TRY(cudaMemcpyAsync(b->tiles, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice, b->st));
    // pageable source: the copy has been staged when the call returns
    return TLB_OK;
}

// the launches of one step of every lattice, entry parity par
static void batch_issue(const tlb_batch *b, int par, cudaStream_t st)
{
    const BatchEntry *E = b->entries[par];
    if (b->D == 2) {
        Launch<2>::step_batch(E, b->tiles, b->ntiles, b->fp16, st, b->cfg.variant);
    } else {
        Launch<3>::moments_batch(E, b->tiles, b->ntiles, b->fp16, st);
        Launch<3>::step_batch(E, b->tiles, b->ntiles, b->fp16, st, b->cfg.variant);
    }
}

// a graph of `depth` steps from entry parity par0; `same` keeps one parity
// for every step (each launch then recomputes the same step: timing only)
static int batch_capture(tlb_batch *b, int par0, int depth, bool same, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < depth; ++s) batch_issue(b, same ? par0 : ((par0 + s) & 1), b->cap);
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess) return fail(TLB_E_CUDA, "batch capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(TLB_E_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    }
    return TLB_OK;
}

extern "C" int tlb_batch_create(tlb_ctx *const *ctxs, int n, const tlb_batch_config *cfg, tlb_batch **out)
{
    NvtxRange range("tlb_batch_create");
    if (!ctxs || n <= 0 || !out) return fail(TLB_E_INVAL, "bad batch arguments");
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!ctxs[k]) return fail(TLB_E_INVAL, "null context in batch");
        if (ctxs[k]->D != ctxs[0]->D) return fail(TLB_E_INVAL, "batched lattices must share the lattice type");
        if (ctxs[k]->p.g_fp16 != ctxs[0]->p.g_fp16)
            return fail(TLB_E_INVAL, "batched lattices must share the g storage");
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == ctxs[k]) return fail(TLB_E_INVAL, "a context appears twice in the batch");
        if (ctxs[k]->stream != ctxs[0]->stream) return fail(TLB_E_INVAL, "batched lattices must share one stream");
    }
    tlb_batch_config c = {};
    c.variant = -1;
    c.tile_order = TLB_ORDER_LATTICE;
    c.graph_depth = 8;
    if (cfg) c = *cfg;
    if (c.tile_order < 0 || c.tile_order > 2) return fail(TLB_E_INVAL, "tile_order must be 0, 1 or 2");
    if (c.graph_depth < 0 || (c.graph_depth & 1)) return fail(TLB_E_INVAL, "graph_depth must be 0 or even");
    if (c.variant < -1 || c.variant > 1) return fail(TLB_E_INVAL, "variant must be -1, 0 or 1");
    tlb_batch *b = new tlb_batch();
    b->ctxs.assign(ctxs, ctxs + n);
    b->D = ctxs[0]->D;
    b->fp16 = ctxs[0]->p.g_fp16;
    b->st = ctxs[0]->stream;
    b->cfg = c;
    b->cfg.us_per_step = 0.0;
    size_t ntiles = batch_tile_order(b, TLB_ORDER_LATTICE).size();
    b->ntiles = (int)ntiles;
    void *ptr;
    int rc = 0;
    for (int par = 0; par < 2 && rc == 0; ++par) {
        if ((rc = dev_alloc(b->owned, &ptr, n * sizeof(BatchEntry), nullptr))) break;
        b->entries[par] = (BatchEntry *)ptr;
    }
    if (rc == 0 && (rc = dev_alloc(b->owned, &ptr, ntiles * sizeof(int4), nullptr)) == 0) b->tiles = (int4 *)ptr;
    if (rc == 0) rc = batch_write_entries(b);
    if (rc == 0) rc = batch_write_tiles(b);
    if (rc == 0 && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        rc = fail(TLB_E_CUDA, "stream creation failed");
    // the table copies are ordered before every launch of the batch (same
    // stream; graphs are replayed on it too): no host synchronisation
    if (rc) {
        if (b->cap) cudaStreamDestroy(b->cap);
        dev_free_all(b->owned);
        delete b;
        return rc;
    }
    *out = b;
    return TLB_OK;
}

extern "C" int tlb_batch_step(tlb_batch *b, int nsteps)
{
    NvtxRange range("tlb_batch_step");
    if (!b || nsteps < 0) return fail(TLB_E_INVAL, "bad batch arguments");
    // the entry parity that matches every context's current buffer; contexts
    // stepped on their own since the entries were written force a rewrite
    const int n = (int)b->ctxs.size();
    int par = (b->ctxs[0]->s.cur + b->base_cur[0]) & 1;
    for (int k = 1; k < n; ++k)
        if (((b->ctxs[k]->s.cur + b->base_cur[k]) & 1) != par) {
            batch_drop_graphs(b);
            int rc = batch_write_entries(b);
            if (rc) return rc;
            par = 0;
            break;
        }
    const int depth = b->cfg.graph_depth;
    int left = nsteps;
    while (left > 0) {
        if (depth > 0 && left >= depth) {
            if (!b->graph[par]) {
                // capture waits for nothing: the graph is replayed on the batch stream
                int rc = batch_capture(b, par, depth, false, &b->graph[par]);
                if (rc) return rc;
            }
            CUDA_TRY(cudaGraphLaunch(b->graph[par], b->st));
            left -= depth;               // even depth: the parity returns to par
        } else {
            batch_issue(b, par, b->st);
            par ^= 1;
            left -= 1;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TLB_E_CUDA, "batched launch: %s", cudaGetErrorString(e));
    const int per = launches_per_step(b->D);
    for (tlb_ctx *c : b->ctxs) {
        if (nsteps & 1) c->s.cur ^= 1;
        c->steps += nsteps;
    }
    b->ctxs[0]->launches += (long long)per * nsteps;
    return TLB_OK;
}

// average time of one step of the batch in configuration c, from `reps`
// replays of a graph of `trial` launches that all recompute the same step
// (the state is left as it was)
static int batch_time(tlb_batch *b, const tlb_batch_config &c, int trial, int reps, double *us)
{
    tlb_batch_config keep = b->cfg;
    b->cfg = c;
    int rc = batch_write_tiles(b);
    const int par = (b->ctxs[0]->s.cur + b->base_cur[0]) & 1;
    cudaGraphExec_t g = nullptr;
    if (rc == 0) rc = batch_capture(b, par, trial, true, &g);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == 0 && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = fail(TLB_E_CUDA, "event creation failed");
    if (rc == 0) {
        cudaStreamSynchronize(b->st);
        cudaGraphLaunch(g, b->cap);                     // warm-up replay
        cudaEventRecord(e0, b->cap);
        for (int r = 0; r < reps; ++r) cudaGraphLaunch(g, b->cap);
        cudaEventRecord(e1, b->cap);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(TLB_E_CUDA, "tuning replay failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *us = 1e3 * ms / (double)(reps * trial);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (g) cudaGraphExecDestroy(g);
    b->cfg = keep;
    return rc;
}

extern "C" int tlb_batch_tune(tlb_batch *b, int reps, tlb_batch_config *chosen)
{
    NvtxRange range("tlb_batch_tune");
    if (!b || reps <= 0) return fail(TLB_E_INVAL, "bad tuning arguments");
    // candidates: register budget (D2Q9), tile order, steps per graph replay;
    // the depth is timed as replays of that many launches, one replay per rep
    const int variants[2] = {0, 1};
    const int nvar = b->D == 2 ? 2 : 1;
    const int depths[3] = {2, 8, 32};
    double best = 1e300;
    tlb_batch_config bestc = b->cfg;
    for (int vi = 0; vi < nvar; ++vi)
        for (int order = 0; order < 3; ++order)
            for (int di = 0; di < 3; ++di) {
                tlb_batch_config c = b->cfg;
                c.variant = b->D == 2 ? variants[vi] : -1;
                c.tile_order = order;
                c.graph_depth = depths[di];
                double us = 0.0;
                int rc = batch_time(b, c, depths[di], std::max(1, reps * 8 / depths[di]), &us);
                if (rc) return rc;
                if (us < best) {
                    best = us;
                    bestc = c;
                }
            }
    bestc.us_per_step = best;
    batch_drop_graphs(b);
    b->cfg = bestc;
    int rc = batch_write_tiles(b);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(b->st));
    if (chosen) *chosen = bestc;
    return TLB_OK;
}

extern "C" int tlb_batch_get_config(const tlb_batch *b, tlb_batch_config *out)
{
    if (!b || !out) return fail(TLB_E_INVAL, "null argument");
    *out = b->cfg;
    return TLB_OK;
}

extern "C" void tlb_batch_destroy(tlb_batch *b)
{
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    batch_drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    dev_free_all(b->owned);
    delete b;
}

// ---------------------------------------------------------------------------
// request server: continuous batching with admission by device-memory budget
// ---------------------------------------------------------------------------
namespace {
double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t ticket;
    tlb_params params;
    std::vector<uint8_t> mask;
    std::vector<double> rho, phi;
    int nsteps, done_steps = 0;
    tlb_ctx *ctx = nullptr;
    tlb_result res;
    size_t bytes = 0;
    std::vector<double> out_rho, out_phi;
};
}  // namespace

struct tlb_server {
    size_t budget;
    int max_active, steps_per_round;
    // stepping streams, one per group (lattice type x g storage): the
    // server's own, so that the groups' rounds overlap on the GPU, or the
    // caller's stream for all of them
    cudaStream_t gstream[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t admit = nullptr;        // initial fields of admitted requests
    bool own_stream = false;
    uint64_t next = 1;
    std::deque<Req *> queue;
    std::vector<Req *> active;
    std::map<uint64_t, Req *> all;
    size_t in_use = 0;
    std::mutex mu;
    // resident batches per group (lattice type x g storage), rebuilt when
    // the group's members change; replaced batches are freed once the
    // stepping stream has passed the event recorded after their last launch
    tlb_batch *batch[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<std::pair<tlb_batch *, cudaEvent_t>> retired;
    int policy = TLB_SCHED_FIFO;         // admission order
    double max_wait_s = 0.0;             // TLB_SCHED_SHORTEST: age after which a request is not overtaken
};

static size_t footprint(const tlb_params &p)
{
    size_t N = (size_t)p.nx * p.ny * p.nz, Q = (size_t)Qof(p.lattice);
    return 2 * Q * N * 4 + 2 * g_bytes(p.lattice, N, p.g_fp16) + N * 9 + (1 << 16);
}

extern "C" int tlb_server_create(size_t budget, int max_active, int steps_per_round, void *stream, tlb_server **out)
{
    if (!out || budget == 0 || max_active <= 0 || steps_per_round <= 0) return fail(TLB_E_INVAL, "bad server arguments");
    tlb_server *s = new tlb_server();
    s->budget = budget;
    s->max_active = max_active;
    s->steps_per_round = steps_per_round;
    s->own_stream = stream == nullptr;
    for (int g = 0; g < 4; ++g) {
        s->gstream[g] = (cudaStream_t)stream;
        if (s->own_stream && cudaStreamCreateWithFlags(&s->gstream[g], cudaStreamNonBlocking) != cudaSuccess) {
            for (int k = 0; k < g; ++k) cudaStreamDestroy(s->gstream[k]);
            delete s;
            return fail(TLB_E_CUDA, "stream creation failed");
        }
    }
    if (cudaStreamCreateWithFlags(&s->admit, cudaStreamNonBlocking) != cudaSuccess) {
        if (s->own_stream)
            for (int g = 0; g < 4; ++g) cudaStreamDestroy(s->gstream[g]);
        delete s;
        return fail(TLB_E_CUDA, "stream creation failed");
    }
    *out = s;
    return TLB_OK;
}

extern "C" int tlb_submit(tlb_server *s, const tlb_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket || !r->rho || !r->phi || r->nsteps < 0) return fail(TLB_E_INVAL, "bad request");
    int rc = validate(r->params);
    if (rc) return rc;
    size_t fp = footprint(r->params);
    if (fp > s->budget) return fail(TLB_E_INVAL, "request needs %zu bytes, budget is %zu", fp, s->budget);
    size_t N = (size_t)r->params.nx * r->params.ny * r->params.nz;
    Req *q = new Req();
    q->params = r->params;
    if (r->mask) q->mask.assign(r->mask, r->mask + N);
    q->rho.assign(r->rho, r->rho + N);
    q->phi.assign(r->phi, r->phi + N);
    q->nsteps = r->nsteps;
    q->bytes = fp;
    std::memset(&q->res, 0, sizeof(q->res));
    q->res.state = TLB_REQ_QUEUED;
    q->res.submit_s = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next++;
    s->queue.push_back(q);
    s->all[q->ticket] = q;
    *ticket = q->ticket;
    return TLB_OK;
}

static void retire(tlb_server *s, Req *q, int status)
{
    if (q->ctx) {
        if (status == TLB_OK) {
            size_t N = (size_t)q->ctx->N;
            q->out_rho.resize(N);
            q->out_phi.resize(N);
            int rc = tlb_get_fields(q->ctx, q->out_rho.data(), q->out_phi.data(), nullptr, nullptr);
            if (rc == TLB_OK) rc = tlb_diagnostics(q->ctx, q->res.mass);
            status = rc;
        }
        tlb_destroy(q->ctx);
        q->ctx = nullptr;
    }
    s->in_use -= q->bytes;
    q->res.status = status;
    q->res.state = status == TLB_OK ? TLB_REQ_DONE : TLB_REQ_FAILED;
    q->res.done_s = now_s();
}

// free the replaced batches whose last launches the stepping stream has passed
static void server_reap(tlb_server *s, bool wait)
{
    std::vector<std::pair<tlb_batch *, cudaEvent_t>> keep;
    for (auto &r : s->retired) {
        if (wait) cudaEventSynchronize(r.second);
        if (cudaEventQuery(r.second) == cudaSuccess) {
            cudaEventDestroy(r.second);
            tlb_batch_destroy(r.first);          // its stream has passed the event: no wait
        } else {
            keep.push_back(r);
        }
    }
    s->retired.swap(keep);
}

static void server_retire_batch(tlb_server *s, int g)
{
    if (!s->batch[g]) return;
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(ev, s->gstream[g]) == cudaSuccess) {
        s->retired.push_back({s->batch[g], ev});
    } else {
        if (ev) cudaEventDestroy(ev);
        tlb_batch_destroy(s->batch[g]);
    }
    s->batch[g] = nullptr;
}

// group of a lattice: lattice type x g storage (one resident batch each)
static int server_group(const tlb_params &p) { return (p.lattice == TLB_D3Q27 ? 1 : 0) + (p.g_fp16 ? 2 : 0); }

// one admitted request: context, solid mask and initial fields on the
// admission stream (the stepping streams keep running), then the context
// moves to its group's stepping stream
static int server_admit_one(tlb_server *s, Req *q)
{
    int rc = tlb_create_ex(&q->params, &q->ctx);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(q->ctx->stream));   // the creation's clears (legacy stream)
    if ((rc = tlb_set_stream(q->ctx, s->admit))) return rc;
    if (!q->mask.empty() && (rc = tlb_set_solid(q->ctx, q->mask.data()))) return rc;
    if ((rc = tlb_init_fields(q->ctx, q->rho.data(), q->phi.data(), nullptr))) return rc;   // synchronises s->admit
    return tlb_set_stream(q->ctx, s->gstream[server_group(q->params)]);
}

// work of a request: node updates still to run
static double req_work(const Req *q)
{
    return (double)q->params.nx * q->params.ny * q->params.nz * (double)(q->nsteps - q->done_steps);
}

// the queued request to admit next: the head (FIFO), or the oldest request
// past max_wait_s, else the least work among those whose memory fits (the
// head when none fits, so that the caller stops admitting)
static std::deque<Req *>::iterator server_pick(tlb_server *s, double now)
{
    if (s->policy == TLB_SCHED_FIFO) return s->queue.begin();
    if (s->max_wait_s > 0.0)
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
            if (now - (*it)->res.submit_s > s->max_wait_s) return it;
    auto best = s->queue.end();
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if (s->in_use + (*it)->bytes > s->budget) continue;
        if (best == s->queue.end() || req_work(*it) < req_work(*best)) best = it;
    }
    return best == s->queue.end() ? s->queue.begin() : best;
}

extern "C" int tlb_server_set_policy(tlb_server *s, int policy, double max_wait_s)
{
    if (!s) return fail(TLB_E_INVAL, "null server");
    if ((policy != TLB_SCHED_FIFO && policy != TLB_SCHED_SHORTEST) || !(max_wait_s >= 0.0))
        return fail(TLB_E_INVAL, "bad policy %d or max_wait_s %g", policy, max_wait_s);
    std::lock_guard<std::mutex> lk(s->mu);
    s->policy = policy;
    s->max_wait_s = max_wait_s;
    return TLB_OK;
}

extern "C" int tlb_server_pump(tlb_server *s)
{
    if (!s) return fail(TLB_E_INVAL, "null server");
    NvtxRange range("tlb_server_pump");
    std::lock_guard<std::mutex> lk(s->mu);
    server_reap(s, false);
    // 1. one round of the active lattices, asynchronously: every group
    //    advances through its resident batch (rebuilt if its members changed)
    int chunk = 0;
    if (!s->active.empty()) {
        chunk = s->steps_per_round;
        for (Req *q : s->active) chunk = std::min(chunk, q->nsteps - q->done_steps);
        std::vector<tlb_ctx *> groups[4];
        for (Req *q : s->active) groups[server_group(q->ctx->p)].push_back(q->ctx);
        for (int g = 0; g < 4; ++g) {
            if (s->batch[g] && s->batch[g]->ctxs != groups[g]) server_retire_batch(s, g);
            if (groups[g].empty()) continue;
            if (!s->batch[g]) {
                int rc = tlb_batch_create(groups[g].data(), (int)groups[g].size(), nullptr, &s->batch[g]);
                if (rc) return rc;
            }
            int rc = tlb_batch_step(s->batch[g], chunk);
            if (rc) return rc;
        }
        for (Req *q : s->active) q->done_steps += chunk;
    }
    // 2. admission while the round runs, in the policy's order while memory
    //    and slots allow; admitted lattices join the next round
    std::vector<Req *> admitted;
    while (!s->queue.empty() && (int)(s->active.size() + admitted.size()) < s->max_active) {
        NvtxRange admit("tlb_server admit");
        auto it = server_pick(s, now_s());
        Req *q = *it;
        if (s->in_use + q->bytes > s->budget) break;
        s->queue.erase(it);
        s->in_use += q->bytes;
        q->res.state = TLB_REQ_RUNNING;
        q->res.start_s = now_s();
        int rc = server_admit_one(s, q);
        q->mask.clear();
        q->rho.clear();
        q->phi.clear();
        if (rc != TLB_OK) { retire(s, q, rc); continue; }
        if (q->nsteps == 0) { retire(s, q, TLB_OK); continue; }
        admitted.push_back(q);
    }
    // 3. retirement of the requests this round completed (their fields are
    //    read after the round; tlb_get_fields waits for their group's stream)
    std::vector<Req *> still;
    for (Req *q : s->active) {
        if (q->done_steps >= q->nsteps) {
            int rc = tlb_sync(q->ctx);
            // the group's batch refers to this context: retire it before the
            // context is freed (a context created later may take its address)
            server_retire_batch(s, server_group(q->ctx->p));
            retire(s, q, rc);
        } else {
            still.push_back(q);
        }
    }
    still.insert(still.end(), admitted.begin(), admitted.end());
    s->active.swap(still);
    return (int)s->active.size();
}

extern "C" int tlb_poll(tlb_server *s, uint64_t ticket, tlb_result *res, double *rho, double *phi)
{
    if (!s || !res) return fail(TLB_E_INVAL, "null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(TLB_E_NOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second;
    *res = q->res;
    if (q->res.state == TLB_REQ_DONE || q->res.state == TLB_REQ_FAILED) {
        if (rho && !q->out_rho.empty()) std::memcpy(rho, q->out_rho.data(), q->out_rho.size() * 8);
        if (phi && !q->out_phi.empty()) std::memcpy(phi, q->out_phi.data(), q->out_phi.size() * 8);
        s->all.erase(it);
        delete q;
    }
    return TLB_OK;
}

extern "C" int tlb_server_stats(tlb_server *s, int *queued, int *active, size_t *bytes)
{
    if (!s) return fail(TLB_E_INVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int)s->queue.size();
    if (active) *active = (int)s->active.size();
    if (bytes) *bytes = s->in_use;
    return TLB_OK;
}

extern "C" void tlb_server_destroy(tlb_server *s)
{
    if (!s) return;
    for (int g = 0; g < 4; ++g) cudaStreamSynchronize(s->gstream[g]);
    for (int g = 0; g < 4; ++g)
        if (s->batch[g]) tlb_batch_destroy(s->batch[g]);
    server_reap(s, true);
    for (Req *q : s->active)
        if (q->ctx) tlb_destroy(q->ctx);
    for (auto &kv : s->all) delete kv.second;
    if (s->admit) cudaStreamDestroy(s->admit);
    if (s->own_stream)
        for (int g = 0; g < 4; ++g) cudaStreamDestroy(s->gstream[g]);
    delete s;
}

// ---------------------------------------------------------------------------
// Allocation-free stepping for callers that cannot allocate device memory
// (no paper counterpart).  The step runs the kernels of tlb_step (the batch
// kernels over a table of one lattice's tiles); their moments, tile table,
// node flags, error word and the two batch entries (one per buffer parity)
// live in one file-scope device array, so the call performs no cudaMalloc,
// cudaFree or other allocation on the device.
// ---------------------------------------------------------------------------
// layout, M = TLB_NOALLOC_MAX_NODES: rho (M floats) | phi (M floats) |
// tiles (M int4: a tile holds at least one node) | flags (M bytes) |
// status word (256 bytes reserved) | entries (2 BatchEntry, 1024 bytes reserved)
constexpr size_t NOALLOC_M = TLB_NOALLOC_MAX_NODES;
constexpr size_t NOALLOC_PHI = NOALLOC_M * 4, NOALLOC_TILES = NOALLOC_M * 8, NOALLOC_FLAGS = NOALLOC_M * 24,
                 NOALLOC_STATUS = NOALLOC_M * 25, NOALLOC_ENTRIES = NOALLOC_M * 25 + 256,
                 NOALLOC_BYTES = NOALLOC_M * 25 + 256 + 1024;
static_assert(2 * sizeof(BatchEntry) <= 1024, "batch entries exceed their reserved bytes");
static_assert(NOALLOC_TILES % 16 == 0 && NOALLOC_ENTRIES % 256 == 0, "scratch alignment");
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
struct NoallocDevice {
    bool ready = false;
    unsigned char *base = nullptr;    // device address of g_noalloc_scratch
    // the geometry whose node flags and ghost list the array holds, and the
    // stream that uploaded them (later work on that stream sees the upload)
    bool have_geom = false;
    int lattice = -1, nx = 0, ny = 0, nz = 0, ntiles = 0;
    cudaStream_t stream = nullptr;
    std::vector<uint8_t> mask;        // empty: no walls
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];
}  // namespace

extern "C" int tlb_step_noalloc(const tlb_params *pin, const uint8_t *mask, float *f, float *f_tmp, void *g,
                                void *g_tmp, int nsteps, void *cuda_stream)
{
    NvtxRange range("tlb_step_noalloc");
    if (!pin || !f || !f_tmp || !g || !g_tmp) return fail(TLB_E_INVAL, "null argument");
    if (nsteps < 0) return fail(TLB_E_INVAL, "nsteps < 0");
    // the same parameter handling as tlb_create_ex: force wetting given by
    // angles takes its strengths from the registered calibration tables
    tlb_params pc = *pin;
    int rc = apply_force_calibration(pc);
    if (rc) return rc;
    const tlb_params *p = &pc;
    rc = validate(*p);
    if (rc) return rc;
    if (p->g_fp16) return fail(TLB_E_UNSUPPORTED, "tlb_step_noalloc takes FP32 g only");
    long long N = (long long)p->nx * p->ny * p->nz;
    if (N > TLB_NOALLOC_MAX_NODES)
        return fail(TLB_E_INVAL, "tlb_step_noalloc handles at most %d nodes (got %lld)", TLB_NOALLOC_MAX_NODES, N);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(TLB_E_UNSUPPORTED, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocDevice &nd = g_noalloc_dev[dev];
    if (!nd.ready) {
        // set-up once per device, with that device current: the device address
        // of the scratch array (its host-side name is not a device address)
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(TLB_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        nd.base = (unsigned char *)ptr;
        nd.ready = true;
    }
    unsigned char *base = nd.base;
    // derived constants: host computation only
    static thread_local tlb_params last_p;
    static thread_local tlb_derived last_d;
    static thread_local bool have_last = false;
    if (!have_last || std::memcmp(&last_p, p, sizeof(tlb_params)) != 0) {
        tlb_derived d;
        rc = derive(*p, d);
        if (rc) return rc;
        last_p = *p;
        last_d = d;
        have_last = true;
    }
    DevParams dp = make_dev(*p, last_d);
    int D = Dof(p->lattice);
    float *rho = (float *)base;
    float *phi = (float *)(base + NOALLOC_PHI);
    int4 *tiles = (int4 *)(base + NOALLOC_TILES);
    uint8_t *type = base + NOALLOC_FLAGS;
    unsigned *status = (unsigned *)(base + NOALLOC_STATUS);
    BatchEntry *entries = (BatchEntry *)(base + NOALLOC_ENTRIES);
    // Node flags (the rules of tlb_set_solid) and the tile table of the
    // lattice.  The array keeps them from the previous call on this device:
    // when the lattice, the sizes, the mask and the stream are the same, that
    // copy is used again and the host pass over the mask skipped (the kernels
    // only read it).  Any other call rebuilds and uploads them.
    bool same = nd.have_geom && nd.lattice == p->lattice && nd.nx == p->nx && nd.ny == p->ny &&
                nd.nz == p->nz && nd.stream == st && (mask == nullptr) == nd.mask.empty() &&
                (mask == nullptr || std::memcmp(mask, nd.mask.data(), (size_t)N) == 0);
    if (!same) {
        nd.have_geom = false;
        std::vector<uint8_t> flags;
        std::vector<int> ghosts;
        node_flags(p->nx, p->ny, p->nz, D, mask, flags, ghosts);
        int TX = D == 2 ? Launch<2>::tile_dims(0) : Launch<3>::tile_dims(0);
        int TY = D == 2 ? Launch<2>::tile_dims(1) : Launch<3>::tile_dims(1);
        int TZ = D == 2 ? Launch<2>::tile_dims(2) : Launch<3>::tile_dims(2);
        std::vector<int4> tl;
        for (int z = 0; z < p->nz; z += TZ)
            for (int y = 0; y < p->ny; y += TY)
                for (int x = 0; x < p->nx; x += TX) tl.push_back(make_int4(0, x, y, z));
        if (tl.size() > NOALLOC_M) return fail(TLB_E_INVAL, "tile table exceeds the scratch array");
        CUDA_TRY(cudaMemcpyAsync(type, flags.data(), (size_t)N, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(tiles, tl.data(), tl.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
        nd.lattice = p->lattice;
        nd.nx = p->nx;
        nd.ny = p->ny;
        nd.nz = p->nz;
        nd.stream = st;
        nd.ntiles = (int)tl.size();
        if (mask) nd.mask.assign(mask, mask + N);
        else nd.mask.clear();
        nd.have_geom = true;
    }
    // one batch entry per buffer parity: parity 0 reads f, g and writes
    // f_tmp, g_tmp; parity 1 the other way round (no tensor maps: the step
    // kernel copies a tile's own populations with cp.async)
    BatchEntry ent[2];
    for (int par = 0; par < 2; ++par) {
        ent[par] = BatchEntry{};
        ent[par].p = dp;
        ent[par].f_in = par ? f_tmp : f;
        ent[par].f_out = par ? f : f_tmp;
        ent[par].g_in = par ? g_tmp : g;
        ent[par].g_out = par ? g : g_tmp;
        ent[par].rho = rho;
        ent[par].phi = phi;
        ent[par].type = type;
        ent[par].status = status;
        for (int k = 0; k < 3; ++k) ent[par].tm[k] = nullptr;
    }
    CUDA_TRY(cudaMemcpyAsync(entries, ent, sizeof(ent), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
    const int ntiles = nd.ntiles;
    int cur = 0;
    for (int k = 0; k < nsteps; ++k) {
        if (D == 2) {
            Launch<2>::step_batch(entries + cur, tiles, ntiles, 0, st);
        } else {
            Launch<3>::moments_batch(entries + cur, tiles, ntiles, 0, st);
            Launch<3>::step_batch(entries + cur, tiles, ntiles, 0, st);
        }
        cur ^= 1;
    }
    if (cur == 1) {
        size_t QN = (size_t)Qof(p->lattice) * (size_t)N;
        CUDA_TRY(cudaMemcpyAsync(f, f_tmp, QN * 4, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(g, g_tmp, QN * 4, cudaMemcpyDeviceToDevice, st));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TLB_E_CUDA, "tlb_step_noalloc launch: %s", cudaGetErrorString(e));
    return TLB_OK;
}
