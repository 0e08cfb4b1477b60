// tlb_internal.h -- shared between the host C-ABI (tlb_api.cu) and the
// per-lattice kernel translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tlb {

// node flags (uint8 per node)
enum : uint8_t {
    TLB_SOLID = 1,      // solid node
    TLB_FIRST = 2,      // fluid node with a solid lattice neighbour (first fluid layer)
    TLB_GHOST = 4,      // solid node with a fluid lattice neighbour (ghost layer)
    TLB_WALLX = 8,      // fluid node with a solid neighbour along +-x
    TLB_WALLY = 16,     // ... along +-y
    TLB_WALLZ = 32,     // ... along +-z
    TLB_NEAR = 64,      // fluid node off the first layer with a first-layer lattice neighbour
};
enum { TLB_WET_FORCE_ = 0 };
#define TLB_WET_FORCE 0
#define TLB_WET_GEOM_EXTRAP 1
#define TLB_WET_GEOM_INTERP 2

// Kernel parameters (FP32 copies of the host FP64 constants).
struct DevParams {
    int nx, ny, nz;
    long long N;
    float lam1, lam2, lam3;
    float chi, inv_chi;
    float a, b, RT, C, Psi0;
    float rho_l, rho_g;
    float inv_drho;      // 1/(rho_l - rho_g)
    float inv_rgl;       // 1/(rho_g - rho_l)
    float krr, kpp, krp;
    float beta, inv_tau_g, Gamma;
    int wetting;
    float cot[3];        // cot(theta_21), cot(theta_31), cot(theta_23)
    float kw_rho, kw_phi;
    int g_fp16;          // g stored as half scaled by 1/chi
    float g_scale, g_unscale;
    int eos;             // TLB_EOS_* (0 Carnahan-Starling, 1 van der Waals, 2 Peng-Robinson)
    float aA;            // Peng-Robinson attraction a A(T)
    int nu_on;           // per-component viscosity: beta from the local mixture
    float nu[3];         // kinematic viscosities of C1, C2, C3
};

// Per-lattice device buffers.
struct DevState {
    float *f[2];          // Q*N each (f - w)
    void *g[2];           // Q*N floats or halves
    float *rho, *phi;     // N
    uint8_t *type;        // N
    int *ghosts;          // ghost-node list
    int nghost;
    int cur;              // index of the current population buffer
    unsigned *status;     // device error flags (STATUS_* bits)
};

// bits of the device status word
enum : unsigned {
    STATUS_DIVERGED = 1u,  // a non-positive density or population was met
    STATUS_TIMEOUT = 2u,   // a bounded wait for a tile's tensor copies gave up
};

// Auxiliary outputs of the step kernel (AUX mode); any may be null.
struct AuxOut {
    float *p0, *mur, *mup, *F[3], *P[6];
};

enum StepMode { MODE_STEP = 0, MODE_INIT = 1, MODE_AUX = 2 };

// Batched execution: one tile -> lattice table entry.
struct BatchEntry {
    DevParams p;
    float *f_in, *f_out;
    void *g_in, *g_out;
    const float *rho, *phi;
    const uint8_t *type;
    unsigned *status;
    // D3Q27 lattices whose strides allow it: tensor maps (device memory) of
    // f_in and g_in (FP32 g) or of its FP32 rest channel and FP16 moving
    // channels, for TMA copies of a tile's own populations; null otherwise
    const void *tm[3];
};

// Launchers implemented per lattice (D = 2: tlb_d2q9.cu, D = 3: tlb_d3q27.cu).
template <int D>
struct Launch {
    static int Q();
    static void moments(const DevParams &p, const DevState &s, cudaStream_t st);
    static void ghosts(const DevParams &p, const DevState &s, cudaStream_t st);
    static void step(const DevParams &p, const DevState &s, int mode, const float *u_init, AuxOut aux,
                     cudaStream_t st);
    static void fields(const DevParams &p, const DevState &s, float *u_out, cudaStream_t st);
    static void diagnostics(const DevParams &p, const DevState &s, double *partials, int nblocks, double *out,
                            cudaStream_t st);
    static int diag_blocks(const DevParams &p);
    // bounds-checked builds: the number of flagged index errors of this lattice
    // type's kernels since the last call (which resets it); 0 otherwise
    static unsigned bounds_errors();
    static void convert_pop(const DevParams &p, const DevState &s, int dir, double *fbuf, double *gbuf,
                            cudaStream_t st);
    // batched: entries[0..n) and a tile table (tile -> entry, tile coords)
    static void moments_batch(const BatchEntry *entries, const int4 *tiles, int ntiles, int g_fp16, cudaStream_t st);
    // variant: D2Q9 register budget, 0 = 3 CTAs/SM (80 registers), 1 = 4 CTAs/SM
    // (64 registers), -1 = 4 CTAs/SM beyond one wave of 3 CTAs/SM; D3Q27 has one
    static void step_batch(const BatchEntry *entries, const int4 *tiles, int ntiles, int g_fp16, cudaStream_t st,
                           int variant = -1);
    static int tile_dims(int a);
};

}  // namespace tlb
