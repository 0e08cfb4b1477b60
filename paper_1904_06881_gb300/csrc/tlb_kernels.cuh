// tlb_kernels.cuh -- kernels and launchers of the ternary ELBM step, templated
// on the dimension D (D2Q9 / D3Q27).  Instantiated once per lattice.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "tlb_device.cuh"

namespace tlb {

// ---- g storage: FP32 [Q][N], or mixed: the rest population g_0 in FP32
// (N floats) followed by the moving populations in FP16, scaled by g_scale
// ([Q-1][N] halves).  g_0 carries phi; the moving ones are small. ----
template <typename GT>
struct GIO;
template <>
struct GIO<float> {
    static __device__ __forceinline__ float ld(const void *p, int i, long long n, const DevParams &q)
    {
        return __ldg((const float *)p + (long long)i * q.N + n);
    }
    static __device__ __forceinline__ void st(void *p, int i, long long n, float v, const DevParams &q)
    {
        ((float *)p)[(long long)i * q.N + n] = v;
    }
};
template <>
struct GIO<__half> {
    static __device__ __forceinline__ float ld(const void *p, int i, long long n, const DevParams &q)
    {
        if (i == 0) return __ldg((const float *)p + n);
        const __half *h = (const __half *)((const char *)p + 4 * q.N);
        return __half2float(h[(long long)(i - 1) * q.N + n]) * q.g_unscale;
    }
    static __device__ __forceinline__ void st(void *p, int i, long long n, float v, const DevParams &q)
    {
        if (i == 0) {
            ((float *)p)[n] = v;
            return;
        }
        __half *h = (__half *)((char *)p + 4 * q.N);
        h[(long long)(i - 1) * q.N + n] = __float2half_rn(v * q.g_scale);
    }
};

template <int D>
struct Tile;
template <>
struct Tile<2> {
    static constexpr int X = 32, Y = 8, Z = 1;
};
template <>
struct Tile<3> {
    static constexpr int X = 8, Y = 8, Z = 4;
};

// periodic wrap of a coordinate at most one period outside [0, n)
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// (node indices fit in 32 bits: a lattice holds at most 2^31 - 1 nodes)
__device__ __forceinline__ int node_near(const DevParams &p, int x, int y, int z)
{
    return (int)chk_node(wrap1(x, p.nx) + p.nx * (wrap1(y, p.ny) + p.ny * wrap1(z, p.nz)), p);
}

// Programmatic dependent launch: a stepping kernel lets the next one be
// scheduled at once and waits for its predecessor's results before reading.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Asynchronous global -> shared copies (sm_80+ cp.async): the node's own
// populations are requested before the tile stages and consumed after them.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Tensor-memory-accelerator copies (cp.async.bulk.tensor): one thread moves a
// tile's box of every direction into shared memory; completion is counted in
// bytes on an mbarrier that the consumers wait on.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the tensor-copy (async) proxy
    asm volatile("fence.mbarrier_init.release.cluster;\n"
                 "fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int c0, int c1, int c2, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];\n"
                 ::"r"(smem_u32(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            unsigned long long *bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];\n"
                 ::"r"(smem_u32(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return done != 0;
}
// waits for the barrier's phase `parity` to complete; false after `ns` nanoseconds
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, unsigned long long ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > ns) return false;
    return true;
}

// dynamic shared memory of the stepping kernel: f (and FP32 g) of the tile's own nodes
template <int D, typename GT>
__host__ __device__ constexpr int stage_bytes()
{
    // f: Q floats; g: Q floats, or g_0 as a float plus Q-1 halves; D3Q27: 128
    // bytes more, to start the area on a 128-byte boundary (tensor copies)
    return Tile<D>::X * Tile<D>::Y * Tile<D>::Z *
               (Lat<D>::Q * 4 + (sizeof(GT) == 4 ? Lat<D>::Q * 4 : 4 + (Lat<D>::Q - 1) * 2)) +
           (D == 3 ? 128 : 0);
}

// ---------------------------------------------------------------------------
// moments: rho = 1 + sum_i (f_i - w_i), phi = sum_i g_i at fluid nodes
// ---------------------------------------------------------------------------
template <int D, typename GT>
__device__ __forceinline__ float2 pop_moments(const DevParams &p, const float *__restrict__ f, const void *g, long long n)
{
    constexpr int Q = Lat<D>::Q;
    float r = 0.f, ph = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        r += __ldg(f + (long long)i * p.N + n);
        ph += GIO<GT>::ld(g, i, n, p);
    }
    return make_float2(1.0f + r, ph);
}

template <int D, typename GT>
__device__ __forceinline__ void moments_node(const DevParams &p, const float *__restrict__ f, const void *g,
                                             const uint8_t *__restrict__ type, float *rho, float *phi, long long n)
{
    constexpr int Q = Lat<D>::Q;
    if (type[n] & TLB_SOLID) {
        if (!(type[n] & TLB_GHOST)) { rho[n] = 0.f; phi[n] = 0.f; }
        return;
    }
    const float2 m = pop_moments<D, GT>(p, f, g, n);
    rho[n] = m.x;
    phi[n] = m.y;
}

template <int D, typename GT>
__global__ void __launch_bounds__(256) moments_kernel(DevParams p, const float *__restrict__ f, const void *g,
                                                      const uint8_t *__restrict__ type, float *rho, float *phi)
{
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < p.N; n += (long long)gridDim.x * blockDim.x)
        moments_node<D, GT>(p, f, g, type, rho, phi, n);
}

template <int D, typename GT>
__global__ void __launch_bounds__(256) moments_batch_kernel(const BatchEntry *__restrict__ E, const int4 *__restrict__ tiles)
{
    pdl_trigger();
    pdl_wait();
    int4 t = tiles[blockIdx.x];
    const BatchEntry &e = E[t.x];
    // the moments need no neighbourhood: the k-th tile of a lattice (in the
    // table's x-fastest order) takes its nodes k*NT .. k*NT + NT - 1 in
    // memory order, so that a warp reads whole 128-byte lines; a lattice has
    // at least N / NT tiles, so every node is covered once
    constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z, NT = TX * TY * TZ;
    const long long ntx = (e.p.nx + TX - 1) / TX, nty = (e.p.ny + TY - 1) / TY;
    const long long k = t.y / TX + ntx * (t.z / TY + nty * (t.w / TZ));
    const long long n = k * NT + threadIdx.x;
    if (n >= e.p.N) return;
    moments_node<D, GT>(e.p, e.f_in, e.g_in, e.type, const_cast<float *>(e.rho), const_cast<float *>(e.phi), n);
}

// ---------------------------------------------------------------------------
// ghost layer (Sec. IV): average over fluid-facing axis directions; ghosts
// with only diagonal fluid neighbours take the mean of those neighbours.
// ---------------------------------------------------------------------------
template <int D, class A>
__device__ void ghost_value(const DevParams &p, const A &acc, int x, int y, int z, float &gr_out, float &gp_out)
{
    constexpr int Q = Lat<D>::Q;
    float sr = 0.f, sp = 0.f;
    int cnt = 0;
    // one copy of the (large) axis code, not one per direction; scalar
    // coordinates (no array indexed by the run-time axis)
#pragma unroll 1
    for (int d = 0; d < 2 * D; ++d) {
        const int a = d >> 1, s = (d & 1) ? 1 : -1;
        const int qx = x + (a == 0 ? s : 0), qy = y + (a == 1 ? s : 0), qz = z + (a == 2 ? s : 0);
        float2 m1;
        if (!acc.get(qx, qy, qz, m1)) continue;
        float gr, gp;
        ghost_axis<D>(p, acc, qx, qy, qz, a, m1, gr, gp);
        sr += gr;
        sp += gp;
        ++cnt;
    }
    if (cnt == 0) {
#pragma unroll 1
        for (int i = 1; i < Q; ++i) {
            float2 m;
            if (!acc.get(x + cc<D>(i, 0), y + cc<D>(i, 1), z + cc<D>(i, 2), m)) continue;
            sr += m.x;
            sp += m.y;
            ++cnt;
        }
    }
    gr_out = cnt > 0 ? sr / (float)cnt : 0.f;
    gp_out = cnt > 0 ? sp / (float)cnt : 0.f;
}

template <int D>
__device__ void ghost_node(const DevParams &p, const uint8_t *__restrict__ type, float *rho, float *phi, long long n)
{
    float gr, gp;
    const int x = (int)(n % p.nx), y = (int)((n / p.nx) % p.ny), z = (int)(n / ((long long)p.nx * p.ny));
    ghost_value<D>(p, NodesGlobal{p, type, rho, phi}, x, y, z, gr, gp);
    rho[n] = gr;
    phi[n] = gp;
}

template <int D>
__global__ void __launch_bounds__(128) ghost_kernel(DevParams p, const uint8_t *__restrict__ type, float *rho, float *phi,
                                                    const int *__restrict__ ghosts, int nghost)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nghost) return;
    ghost_node<D>(p, type, rho, phi, ghosts[k]);
}

// ---------------------------------------------------------------------------
// Node thermodynamics from a shared-memory tile of rho, phi (halo 2).
// ---------------------------------------------------------------------------
template <int D>
struct Thermo {
    float gr[3], gp[3], lr, lp;
    Bulk b;
    float mur, mup;
    float P[6];     // xx yy zz xy xz yz
};

template <int D, int RX, int RY>
__device__ __forceinline__ Thermo<D> node_thermo(const DevParams &p, const float2 *srp, int hx,
                                                 int hy, int hz)
{
    constexpr int Q = Lat<D>::Q;
    Thermo<D> t;
    int c0 = hx + RX * (hy + RY * hz);
    const float2 m0 = srp[c0];
    float r0 = m0.x, p0v = m0.y;
#pragma unroll
    for (int a = 0; a < 3; ++a) { t.gr[a] = 0.f; t.gp[a] = 0.f; }
    t.lr = 0.f;
    t.lp = 0.f;
    // grad Q = 3 sum w_i c_i Q(x + c_i); lap Q = 6 sum w_i (Q(x + c_i) - Q(x))
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        int m = (hx + cc<D>(i, 0)) + RX * ((hy + cc<D>(i, 1)) + RY * (hz + cc<D>(i, 2)));
        const float2 mm = srp[m];
        float rm = mm.x, pm = mm.y;
        float w3 = 3.0f * wt<D>(i);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (cc<D>(i, a) != 0) {
                t.gr[a] += (float)cc<D>(i, a) * w3 * rm;
                t.gp[a] += (float)cc<D>(i, a) * w3 * pm;
            }
        }
        t.lr += 2.0f * w3 * (rm - r0);
        t.lp += 2.0f * w3 * (pm - p0v);
    }
    t.b = bulk_terms(p, r0, p0v);
    t.mur = t.b.murB - p.krr * t.lr - p.krp * t.lp;
    t.mup = t.b.mupB - p.kpp * t.lp - p.krp * t.lr;
    float g2r = 0.f, g2p = 0.f, grp = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        g2r += t.gr[a] * t.gr[a];
        g2p += t.gp[a] * t.gp[a];
        grp += t.gr[a] * t.gp[a];
    }
    float iso = t.b.p0 - p.krr * (r0 * t.lr + 0.5f * g2r) - p.kpp * (p0v * t.lp + 0.5f * g2p) -
                p.krp * (r0 * t.lp + p0v * t.lr + grp);
    constexpr int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        int a = pa[k], b = pb[k];
        float v = 0.f;
        if (a < D && b < D) {
            v = p.krr * t.gr[a] * t.gr[b] + p.kpp * t.gp[a] * t.gp[b] + p.krp * (t.gr[a] * t.gp[b] + t.gp[a] * t.gr[b]);
            if (a == b) v += iso;
        }
        t.P[k] = v;
    }
    return t;
}

template <int D>
__host__ __device__ constexpr int NQC() { return D == 2 ? 3 : 6; }

// index into the Q-tensor components stored per node: 2D {xx, yy, xy}, 3D {xx, yy, zz, xy, xz, yz}
template <int D>
__device__ __forceinline__ int qcomp(int a, int b)
{
    if (a == b) return a;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    if (D == 2) return 2;
    return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// Flag test and moments of a node outside the tile region: from the flag
// array and the node's populations.  Out of line, so that the several call
// sites of the ghost-layer code share one copy of the index arithmetic.
template <int D, typename GT>
__device__ __noinline__ bool node_far(const DevParams &p, const uint8_t *__restrict__ type, const float *__restrict__ f,
                                      const void *g, int x, int y, int z, float2 &m)
{
    const long long n = node_of(p, x, y, z);
    if (type[n] & TLB_SOLID) return false;
    m = pop_moments<D, GT>(p, f, g, n);
    return true;
}

// Node accessor of the ghost pass of a D2Q9 tile that sums its own moments:
// node flags and moments from a box in shared memory (the tile + halo 2 and a
// margin that holds the samples of the ghost layer), else from the flag
// array and the node's populations.  (ox, oy) is the box's first node.
template <int D, typename GT, int BX, int BY>
struct NodesBox {
    const DevParams &p;
    const uint8_t *type;
    const float *f;
    const void *g;
    const uint8_t *bt;
    const float *br, *bp;
    int ox, oy;
    __device__ __forceinline__ bool get(int x, int y, int, float2 &m) const
    {
        const int lx = x - ox, ly = y - oy;
        if ((unsigned)lx < (unsigned)BX && (unsigned)ly < (unsigned)BY) {
            const int k = lx + BX * ly;
            if (bt[k] & TLB_SOLID) return false;
            m = make_float2(br[k], bp[k]);
            return true;
        }
        return node_far<D, GT>(p, type, f, g, x, y, 0, m);
    }
};

// ---------------------------------------------------------------------------
// The fused step kernel.  One CTA = one tile of TX x TY x TZ nodes.
// ASYNC: the node's own populations are staged by cp.async before stage A.
// FUSED (D2Q9): stage A sums rho, phi of the tile + halo 2 from the
// populations itself (no moments pass before the step) and keeps the tile's
// own populations in shared memory.
// ---------------------------------------------------------------------------
template <int D, typename GT, int MODE, bool ASYNC = false, bool FUSED = false, bool FIRSTNB = (D == 3)>
__device__ __forceinline__ void step_tile(const DevParams &p, const float *__restrict__ f_in, float *__restrict__ f_out,
                                          const void *g_in, void *g_out, const float *__restrict__ rho,
                                          const float *__restrict__ phi, const uint8_t *__restrict__ type,
                                          unsigned *status, int x0, int y0, int z0, const float *__restrict__ u_init,
                                          const AuxOut &aux, const void *const *tm = nullptr)
{
    constexpr int Q = Lat<D>::Q;
    constexpr int TX = Tile<D>::X, TY = Tile<D>::Y, TZ = Tile<D>::Z;
    constexpr int RX = TX + 4, RY = TY + 4, RZ = (D == 3) ? TZ + 4 : 1;
    constexpr int SX = TX + 2, SY = TY + 2, SZ = (D == 3) ? TZ + 2 : 1;
    constexpr int NR = RX * RY * RZ, NS = SX * SY * SZ;
    constexpr int HZ2 = (D == 3) ? 2 : 0, HZ1 = (D == 3) ? 1 : 0;
    constexpr int NC = NQC<D>();
    // rho, phi of the tile + halo 2, interleaved (one 8-byte access per node)
    __shared__ float2 srp[NR];
    // Q = rho c_s^2 I - P of the tile + halo 1: D2Q9 one array per component;
    // D3Q27 per node as {xx, yy, zz, xy} and {xz, yz}, so that the force
    // stencil reads a neighbour's tensor with two vector loads
    __shared__ float sQ[D == 2 ? NC : 1][D == 2 ? NS : 1];
    __shared__ float4 sQa[D == 3 ? NS : 1];
    __shared__ float2 sQb[D == 3 ? NS : 1];
    // component c (qcomp order) of Q at slot m
    auto qc = [&](int c, int m) -> float {
        if constexpr (D == 2) return sQ[c][m];
        else return c == 0 ? sQa[m].x : c == 1 ? sQa[m].y : c == 2 ? sQa[m].z : c == 3 ? sQa[m].w
                    : c == 4 ? sQb[m].x : sQb[m].y;
    };
    __shared__ float smu[NS];
    __shared__ uint8_t stype[NS];
    __shared__ uint8_t srt[NR];               // node flags of the tile + halo 2
    // FUSED tiles with ghost nodes: flags and moments of the tile + halo 2
    // widened by EM nodes, the reach of the ghost layer (for theta in
    // [20, 160] deg a ghost node's samples lie at most 3 nodes along the wall
    // and 1 across from it; farther nodes are read from global memory)
    constexpr int EM = 3, BX = RX + 2 * EM, BY = RY + 2 * EM, NB = FUSED ? BX * BY : 1;
    __shared__ float brho[NB], bphi[NB];
    __shared__ uint8_t btyp[NB];
    // FUSED: the region's ghost slots, one per thread in the ghost pass
    __shared__ short glist[FUSED ? NR : 1];
    __shared__ int nghost;
    const int tid = threadIdx.x;
    constexpr int NT = TX * TY * TZ;
    // ASYNC: f[Q][NT], then FP32 g[Q][NT] (or the FP32 rest channel [NT] and
    // the FP16 moving channels [Q-1][NT]); D3Q27: from the first 128-byte
    // boundary of the dynamic area (tensor-copy destinations)
    extern __shared__ __align__(16) float stage_raw[];
    float *const stage = D == 3 ? stage_raw + (((128u - (smem_u32(stage_raw) & 127u)) & 127u) >> 2) : stage_raw;
    // ASYNC with tensor maps: the copies' completion barrier
    __shared__ unsigned long long tma_bar;
    // tensor copies need the staging area 128-byte aligned (checked, uniform per CTA)
    const bool use_tma = ASYNC && tm != nullptr && tm[0] != nullptr && (smem_u32(stage) & 127u) == 0;

    // Region slots are filled for coordinates below n + 2 (n + 1 for the flags)
    // along each axis: the tile's nodes use no farther neighbours, and
    // node_near wraps one period only.
    if constexpr (FUSED) {
        static_assert(D == 2 && !ASYNC, "summed moments: D2Q9 tiles");
        // Stage A1: thread tid sums its own node (tile slot tid) and, for
        // tid < NR - NT, one node of the halo ring: rows 0-1 and RY-2..RY-1,
        // then the two columns on either side of rows 2..RY-3.
        constexpr int NH = NR - NT;
        static_assert(NH == 4 * RX + 4 * TY && NT == 256, "halo ring of a 32 x 8 tile");
        int kl[2], kx[2], ky[2];
        kx[0] = 2 + tid % TX;
        ky[0] = 2 + tid / TX;
        const bool has_h = tid < NH;
        {
            const int h = has_h ? tid : 0;
            if (h < 2 * RX) { kx[1] = h % RX; ky[1] = h / RX; }
            else if (h < 4 * RX) { kx[1] = (h - 2 * RX) % RX; ky[1] = RY - 2 + (h - 2 * RX) / RX; }
            else {
                const int c = (h - 4 * RX) & 3;
                kx[1] = c < 2 ? c : TX + c;
                ky[1] = 2 + ((h - 4 * RX) >> 2);
            }
        }
        float fa[2][Q], ga[2][Q];
        __half gh[2][Q];                     // FP16 storage: the raw moving populations
        int na[2];
        bool in[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            kl[s] = kx[s] + RX * ky[s];
            const int X = x0 - 2 + kx[s], Y = y0 - 2 + ky[s];
            in[s] = (s == 0 || has_h) && X < p.nx + 2 && Y < p.ny + 2;
            na[s] = in[s] ? node_near(p, X, Y, 0) : 0;
        }
        // issue both nodes' loads before any sum
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                fa[s][i] = in[s] ? __ldg(f_in + na[s] + (long long)i * p.N) : 0.f;
                if (sizeof(GT) == 4 || i == 0) {
                    ga[s][i] = in[s] ? __ldg((const float *)g_in + na[s] + (long long)i * p.N) : 0.f;
                } else {
                    // the value GIO<__half>::ld returns, from one load of the raw half
                    const __half *hb = (const __half *)((const char *)g_in + 4 * p.N);
                    gh[s][i] = in[s] ? hb[(long long)(i - 1) * p.N + na[s]] : __float2half_rn(0.f);
                    ga[s][i] = __half2float(gh[s][i]) * p.g_unscale;
                }
            }
        if (x0 + kx[0] - 2 < p.nx && y0 + ky[0] - 2 < p.ny) {
            // the node's own populations for stage C, in the staging layout
#pragma unroll
            for (int i = 0; i < Q; ++i) stage[i * NT + tid] = fa[0][i];
            if (sizeof(GT) == 4) {
#pragma unroll
                for (int i = 0; i < Q; ++i) stage[(Q + i) * NT + tid] = ga[0][i];
            } else {
                stage[Q * NT + tid] = ga[0][0];
                __half *s16 = reinterpret_cast<__half *>(&stage[(Q + 1) * NT]);
#pragma unroll
                for (int i = 1; i < Q; ++i) s16[(i - 1) * NT + tid] = gh[0][i];
            }
        }
        bool ghost = false;
        if (tid == 0) nghost = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && !has_h) break;
            float r = 0.f, ph = 0.f;
            uint8_t t = TLB_SOLID;
            if (in[s]) {
                t = __ldg(type + na[s]);
                ghost |= (t & TLB_GHOST) != 0;
                if (!(t & TLB_SOLID)) {
                    // the summation order of the moments kernel
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        r += fa[s][i];
                        ph += ga[s][i];
                    }
                    r = 1.0f + r;
                }
            }
            srp[kl[s]] = make_float2(r, ph);
            srt[kl[s]] = t;
        }
        // Stage A2: the ghost layer of Sec. IV from the fluid moments
        if (__syncthreads_or(ghost)) {
            // list the ghost slots (in any order: each ghost value depends on
            // the box alone), so that no thread takes more than one of them
            for (int k = tid; k < NR; k += NT)
                if (srt[k] & TLB_GHOST) glist[atomicAdd(&nghost, 1)] = (short)k;
            // the box: region slots copied (where filled) ...
            for (int k = tid; k < NR; k += NT) {
                const int lx = k % RX, ly = k / RX, kb = (lx + EM) + BX * (ly + EM);
                const int X = x0 - 2 + lx, Y = y0 - 2 + ly;
                if (X < p.nx + 2 && Y < p.ny + 2) {
                    btyp[kb] = srt[k];
                    brho[kb] = srp[k].x;
                    bphi[kb] = srp[k].y;
                } else {                      // lattices narrower than a tile
                    const long long n = node_of(p, X, Y, 0);
                    const uint8_t t = __ldg(type + n);
                    const float2 m = pop_moments<D, GT>(p, f_in, g_in, n);
                    btyp[kb] = t;
                    brho[kb] = (t & TLB_SOLID) ? 0.f : m.x;
                    bphi[kb] = (t & TLB_SOLID) ? 0.f : m.y;
                }
            }
            // ... and the margin summed from the populations: at most two
            // nodes per thread, all loads issued before the sums.  Margin
            // index h: rows above, rows below, then the columns either side.
            constexpr int NM = BX * BY - RX * RY;
            static_assert(NM <= 2 * NT, "margin of two nodes per thread");
            int kb[2];
            long long nm[2];
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int h = (tid + NT * j < NM) ? tid + NT * j : 0;
                int bx, by;
                if (h < EM * BX) { bx = h % BX; by = h / BX; }
                else if (h < 2 * EM * BX) { bx = (h - EM * BX) % BX; by = BY - EM + (h - EM * BX) / BX; }
                else {
                    const int c = (h - 2 * EM * BX) % (2 * EM);
                    bx = c < EM ? c : RX + c;
                    by = EM + (h - 2 * EM * BX) / (2 * EM);
                }
                kb[j] = bx + BX * by;
                nm[j] = node_of(p, x0 - 2 - EM + bx, y0 - 2 - EM + by, 0);
            }
            const uint8_t t0 = __ldg(type + nm[0]), t1 = __ldg(type + nm[1]);
            const float2 m0 = pop_moments<D, GT>(p, f_in, g_in, nm[0]);
            const float2 m1 = pop_moments<D, GT>(p, f_in, g_in, nm[1]);
            if (tid < NM) {
                btyp[kb[0]] = t0;
                brho[kb[0]] = (t0 & TLB_SOLID) ? 0.f : m0.x;
                bphi[kb[0]] = (t0 & TLB_SOLID) ? 0.f : m0.y;
            }
            if (tid + NT < NM) {
                btyp[kb[1]] = t1;
                brho[kb[1]] = (t1 & TLB_SOLID) ? 0.f : m1.x;
                bphi[kb[1]] = (t1 & TLB_SOLID) ? 0.f : m1.y;
            }
            __syncthreads();
            const NodesBox<D, GT, BX, BY> acc{p, type, f_in, g_in, btyp, brho, bphi, x0 - 2 - EM, y0 - 2 - EM};
            for (int j = tid; j < nghost; j += NT) {
                const int k = glist[j];
                float gr, gp;
                ghost_value<D>(p, acc, x0 - 2 + k % RX, y0 - 2 + k / RX, 0, gr, gp);
                srp[k] = make_float2(gr, gp);
            }
            __syncthreads();      // the ghost values, before stage B reads them
        }
    } else {
        // Stage A: rho, phi and flags of the tile + halo 2, all of a thread's
        // slots loaded in one round (loads issued before use); then the ghost
        // layer of Sec. IV from the fluid moments (the moments pass leaves
        // ghost nodes alone)
        constexpr int PER = (NR + NT - 1) / NT;
        float lr[PER], lp[PER];
        uint8_t lt[PER];
        bool ghost = false;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int k = tid + NT * j;
            const int X = x0 - 2 + k % RX, Y = y0 - 2 + (k / RX) % RY, Z = z0 - HZ2 + k / (RX * RY);
            const bool in = k < NR && X < p.nx + 2 && Y < p.ny + 2 && Z < p.nz + 2;
            const int n = in ? node_near(p, X, Y, Z) : 0;
            lt[j] = in ? __ldg(type + n) : (uint8_t)TLB_SOLID;
            lr[j] = in ? __ldg(rho + n) : 0.f;
            lp[j] = in ? __ldg(phi + n) : 0.f;
        }
        // the node's own populations for stage C, requested after the loads stage A
        // waits on (they would queue ahead of them otherwise)
        if (use_tma) {
            // one thread: a box of TX x TY x TZ nodes x all directions per array
            // (x0 is a multiple of 8 nodes: 16-byte aligned inner coordinate)
            if (tid == 0) {
                mbar_init(&tma_bar, 1);
                const unsigned bytes = (unsigned)(Q * NT * 4) +
                                       (sizeof(GT) == 4 ? (unsigned)(Q * NT * 4) : (unsigned)(NT * 4 + (Q - 1) * NT * 2));
#ifdef TLB_TEST_TMA_TIMEOUT
                // test builds only: the barrier expects 16 bytes more than the
                // copies send, so its wait runs out and the timeout path runs
                mbar_expect_tx(&tma_bar, bytes + 16u);
#else
                mbar_expect_tx(&tma_bar, bytes);
#endif
                tma_load_4d(&stage[0], tm[0], x0, y0, z0, 0, &tma_bar);
                if (sizeof(GT) == 4) {
                    tma_load_4d(&stage[Q * NT], tm[1], x0, y0, z0, 0, &tma_bar);
                } else {
                    tma_load_3d(&stage[Q * NT], tm[1], x0, y0, z0, &tma_bar);
                    tma_load_4d(&stage[(Q + 1) * NT], tm[2], x0, y0, z0, 0, &tma_bar);
                }
            }
        } else if (ASYNC) {
            const int ax = x0 + tid % TX, ay = y0 + (tid / TX) % TY, az = z0 + tid / (TX * TY);
            if (ax < p.nx && ay < p.ny && az < p.nz) {
                const long long an = (long long)ax + (long long)p.nx * ((long long)ay + (long long)p.ny * az);
#pragma unroll
                for (int i = 0; i < Q; ++i) cp_async4(&stage[i * NT + tid], f_in + (long long)i * p.N + an);
                if (sizeof(GT) == 4) {
#pragma unroll
                    for (int i = 0; i < Q; ++i)
                        cp_async4(&stage[(Q + i) * NT + tid], (const float *)g_in + (long long)i * p.N + an);
                } else {
                    cp_async4(&stage[Q * NT + tid], (const float *)g_in + an);
                    // the FP16 moving populations of two x-neighbours share a 4-byte
                    // word (nx even): the even thread of each pair copies it
                    if ((p.nx & 1) == 0 && (tid & 1) == 0) {
                        const char *h = (const char *)g_in + 4 * p.N;
                        __half *s16 = reinterpret_cast<__half *>(&stage[(Q + 1) * NT]);
#pragma unroll
                        for (int i = 1; i < Q; ++i)
                            cp_async4(&s16[(i - 1) * NT + tid], h + 2 * ((long long)(i - 1) * p.N + an));
                    }
                }
            }
            cp_async_commit();
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int k = tid + NT * j;
            if (k >= NR) break;
            srt[k] = lt[j];
            srp[k] = make_float2(lr[j], lp[j]);
            ghost |= (lt[j] & TLB_GHOST) != 0;
        }
        if (ghost) {
            const NodesGlobal acc{p, type, rho, phi};
#pragma unroll 1
            for (int k = tid; k < NR; k += NT) {
                if (!(srt[k] & TLB_GHOST)) continue;      // unfilled slots hold TLB_SOLID alone
                float gr, gp;
                ghost_value<D>(p, acc, x0 - 2 + k % RX, y0 - 2 + (k / RX) % RY, z0 - HZ2 + k / (RX * RY), gr, gp);
                srp[k] = make_float2(gr, gp);
            }
        }
        __syncthreads();
    }
    // slot stride of the tile + halo 1 loops: the compile-time thread count
    // for D2Q9 (the loops unroll; measured faster), the run-time one for
    // D3Q27 (the unrolled loops measured 3 % slower)
    const int KSTEP = D == 2 ? NT : (int)blockDim.x;
    // Stage B: Q = rho c_s^2 I - P and mu_phi at every fluid node of the tile
    // + halo 1, with the node flags of the tile + halo 1 (from those of the
    // region; read by stage C after the barrier that follows)
    for (int k = tid; k < NS; k += KSTEP) {
        const int lx = k % SX, ly = (k / SX) % SY, lz = k / (SX * SY);
        const int X = x0 - 1 + lx, Y = y0 - 1 + ly, Z = z0 - HZ1 + lz;
        const uint8_t tk = (X >= p.nx + 1 || Y >= p.ny + 1 || Z >= p.nz + 1)
                               ? (uint8_t)TLB_SOLID
                               : srt[(lx + 1) + RX * ((ly + 1) + RY * (lz + (D == 3 ? 1 : 0)))];
        stype[k] = tk;
        if (tk & TLB_SOLID) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                if constexpr (D == 2) sQ[c][k] = 0.f;
            }
            if constexpr (D == 3) {
                sQa[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                sQb[k] = make_float2(0.f, 0.f);
            }
            smu[k] = 0.f;
            continue;
        }
        Thermo<D> t = node_thermo<D, RX, RY>(p, srp, lx + 1, ly + 1, lz + (D == 3 ? 1 : 0));
        float r0 = srp[(lx + 1) + RX * ((ly + 1) + RY * (lz + (D == 3 ? 1 : 0)))].x;
        if constexpr (D == 2) {
            sQ[0][k] = r0 * (1.0f / 3.0f) - t.P[0];
            sQ[1][k] = r0 * (1.0f / 3.0f) - t.P[1];
            sQ[2][k] = -t.P[3];
        } else {
            sQa[k] = make_float4(r0 * (1.0f / 3.0f) - t.P[0], r0 * (1.0f / 3.0f) - t.P[1],
                                 r0 * (1.0f / 3.0f) - t.P[2], -t.P[3]);
            sQb[k] = make_float2(-t.P[4], -t.P[5]);
        }
        smu[k] = t.mup;
    }
    // every thread's staged copies complete before the barrier, so each thread
    // may read copies made by another (the FP16 pairs) and none is pending
    // when a thread leaves
    if (use_tma) {
        // every thread waits on the copies' barrier (its completion makes the
        // tensor copies visible to the waiting thread), at most one second; a
        // CTA whose copies did not land flags the lattice, waits once more
        // (bounded) so that no copy is left in flight, and skips the tile
        bool lost = !mbar_wait_bounded(&tma_bar, 0, 1000000000ull);
        if (__syncthreads_or(lost)) {
            if (tid == 0) atomicOr(status, STATUS_TIMEOUT);
            if (lost) mbar_wait_bounded(&tma_bar, 0, 1000000000ull);
            return;
        }
    } else {
        if (ASYNC) cp_async_wait_all();
        __syncthreads();
    }

    // Stage C: one node per thread
    const int tx = tid % TX, ty = (tid / TX) % TY, tz = tid / (TX * TY);
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    if (x >= p.nx || y >= p.ny || z >= p.nz) return;
    const int sx = tx + 1, sy = ty + 1, sz = tz + HZ1;
    const int sc = sx + SX * (sy + SY * sz);
    const uint8_t tc = stype[sc];
    // node indices fit in 32 bits (lattices hold at most 2^31 - 1 nodes)
    const int n = x + p.nx * (y + p.ny * z);
    if (tc & TLB_SOLID) return;
    // push-streaming store addresses: the node index plus one offset per axis
    // and sign (periodic wrap included), formed once per node
    const int oxm = x == 0 ? p.nx - 1 : -1, oxq = x == p.nx - 1 ? 1 - p.nx : 1;
    const int oym = (y == 0 ? p.ny - 1 : -1) * p.nx;
    const int oyq = (y == p.ny - 1 ? 1 - p.ny : 1) * p.nx;
    const int oz = D == 3 ? p.nx * p.ny : 0;
    const int ozm = D == 3 ? (z == 0 ? p.nz - 1 : -1) * oz : 0;
    const int ozq = D == 3 ? (z == p.nz - 1 ? 1 - p.nz : 1) * oz : 0;
    auto nbr = [&](int cx, int cy, int cz) -> int {
        int m = n;
        if (cx != 0) m += cx > 0 ? oxq : oxm;
        if (cy != 0) m += cy > 0 ? oyq : oym;
        if (D == 3 && cz != 0) m += cz > 0 ? ozq : ozm;
        return (int)chk_node(m, p);
    };
    const float2 rph = srp[(sx + 1) + RX * ((sy + 1) + RY * (sz + (D == 3 ? 1 : 0)))];
    const float r = rph.x, ph = rph.y;

    // force F = div(rho c_s^2 I - P) with the wall rules (Sec. IV)
    float F[3] = {0.f, 0.f, 0.f};
    if (!(tc & TLB_FIRST)) {
        // no solid node within one link: the isotropic stencil, one pass over the neighbours
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int m = (sx + cc<D>(i, 0)) + SX * ((sy + cc<D>(i, 1)) + SY * (sz + cc<D>(i, 2)));
            const float w3 = 3.0f * wt<D>(i);
            float q[NC];
            if constexpr (D == 2) {
#pragma unroll
                for (int c = 0; c < NC; ++c) q[c] = sQ[c][m];
            } else {
                const float4 qa = sQa[m];
                const float2 qb = sQb[m];
                q[0] = qa.x; q[1] = qa.y; q[2] = qa.z; q[3] = qa.w; q[4] = qb.x; q[5] = qb.y;
            }
#pragma unroll
            for (int a = 0; a < D; ++a) {
                float acc = 0.f;
#pragma unroll
                for (int gdir = 0; gdir < D; ++gdir)
                    if (cc<D>(i, gdir) != 0) acc += (float)cc<D>(i, gdir) * q[qcomp<D>(a, gdir)];
                F[a] += w3 * acc;
            }
        }
    } else {
        bool wall[3] = {(tc & TLB_WALLX) != 0, (tc & TLB_WALLY) != 0, (tc & TLB_WALLZ) != 0};
#pragma unroll
        for (int gdir = 0; gdir < D; ++gdir) {
            if (wall[gdir]) {
                // one-sided along a wall axis: fluid-side differences, doubled
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    if (cc<D>(i, gdir) == 0) continue;
                    int m = (sx + cc<D>(i, 0)) + SX * ((sy + cc<D>(i, 1)) + SY * (sz + cc<D>(i, 2)));
                    if (stype[m] & TLB_SOLID) continue;
                    float wc = 6.0f * wt<D>(i) * (float)cc<D>(i, gdir);
#pragma unroll
                    for (int a = 0; a < D; ++a) F[a] += wc * (qc(qcomp<D>(a, gdir), m) - qc(qcomp<D>(a, gdir), sc));
                }
            } else {
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    if (cc<D>(i, gdir) == 0) continue;
                    int cx = cc<D>(i, 0), cy = cc<D>(i, 1), cz = cc<D>(i, 2);
                    int m = (sx + cx) + SX * ((sy + cy) + SY * (sz + cz));
                    if (stype[m] & TLB_SOLID) {
                        // mirror image across the wall axes, else the node itself
                        if (wall[0]) cx = -cx;
                        if (wall[1]) cy = -cy;
                        if (D == 3 && wall[2]) cz = -cz;
                        int mm = (sx + cx) + SX * ((sy + cy) + SY * (sz + cz));
                        m = (stype[mm] & TLB_SOLID) ? sc : mm;
                    }
                    float wc = 3.0f * wt<D>(i) * (float)cc<D>(i, gdir);
#pragma unroll
                    for (int a = 0; a < D; ++a) F[a] += wc * qc(qcomp<D>(a, gdir), m);
                }
            }
        }
    }
    // wetting force of method 1 (Eq. forceBC) on fluid nodes off the first layer
    if (p.wetting == TLB_WET_FORCE && (tc & TLB_NEAR) && (p.kw_rho != 0.f || p.kw_phi != 0.f)) {
        float rrel = (r - p.rho_g) * p.inv_drho;
        float amp = rrel * (p.kw_rho + ph * p.inv_chi * p.kw_phi);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            int m = (sx + cc<D>(i, 0)) + SX * ((sy + cc<D>(i, 1)) + SY * (sz + cc<D>(i, 2)));
            if (!(stype[m] & TLB_FIRST)) continue;
#pragma unroll
            for (int a = 0; a < D; ++a) F[a] += amp * wt<D>(i) * (float)cc<D>(i, a);
        }
    }
    const float mup = smu[sc];

    if (MODE == MODE_AUX) {
        Thermo<D> t = node_thermo<D, RX, RY>(p, srp, sx + 1, sy + 1, sz + (D == 3 ? 1 : 0));
        if (aux.p0) aux.p0[n] = t.b.p0;
        if (aux.mur) aux.mur[n] = t.mur;
        if (aux.mup) aux.mup[n] = t.mup;
        for (int a = 0; a < 3; ++a)
            if (aux.F[a]) aux.F[a][n] = (a < D) ? F[a] : 0.f;
        for (int k = 0; k < 6; ++k)
            if (aux.P[k]) aux.P[k][n] = t.P[k];
        return;
    }

    const float inv_r = 1.0f / r;
    if (MODE == MODE_INIT) {
        // f = f^eq(rho, v - F/(2 rho)), g = g^eq(phi, v, mu_phi) at the node itself
        float v[3] = {0.f, 0.f, 0.f}, ub[3];
#pragma unroll
        for (int a = 0; a < D; ++a) {
            v[a] = u_init ? u_init[(long long)a * p.N + n] : 0.f;
            ub[a] = v[a] - 0.5f * F[a] * inv_r;
        }
        Fac fu[3];
#pragma unroll
        for (int a = 0; a < D; ++a) fu[a] = eq_factors(ub[a]);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float e = r;
#pragma unroll
            for (int a = 0; a < D; ++a) e *= fac_of(fu[a], cc<D>(i, a));
            f_out[(long long)i * p.N + n] = e - wt<D>(i);
        }
        float v2 = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) v2 += v[a] * v[a];
        float gsum = 0.f;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            float cv = 0.f;
#pragma unroll
            for (int a = 0; a < D; ++a) cv += (float)cc<D>(i, a) * v[a];
            float ge = wt<D>(i) * (3.0f * p.Gamma * mup + 3.0f * ph * cv + 4.5f * ph * cv * cv - 1.5f * ph * v2);
            gsum += ge;
            GIO<GT>::st(g_out, i, n, ge, p);
        }
        GIO<GT>::st(g_out, 0, n, ph - gsum, p);
        return;
    }

    // ---- ELBM collision of f (Eqs. ELBMequation, ELBMForcingExactDiff, EntropyEquation) ----
    // fp holds f~ = f - w on load and the mirror state f' after the pass below.
    float fp[Q], dl[Q];
    float j[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float fi = (ASYNC || FUSED) ? stage[i * NT + tid] : __ldg(f_in + (long long)i * p.N + n);
        fp[i] = fi;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (cc<D>(i, a) != 0) j[a] += (float)cc<D>(i, a) * fi;
    }
    float u[3], ud[3], v[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        u[a] = j[a] * inv_r;
        float du = F[a] * inv_r;          // delta u = F dt / rho
        ud[a] = u[a] + du;
        v[a] = u[a] + 0.5f * du;          // fluid velocity
    }
    Fac fu[3], fd[3];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        fu[a] = eq_factors(u[a]);
        fd[a] = eq_factors(ud[a]);
    }
    // The relaxation D_i = f^eq_i(u) - f_i carries no mass or momentum and the
    // forcing term F_i = f^eq_i(u+du) - f^eq_i(u) carries mass 0 and momentum F.
    // In FP32 the rest population closes the mass balances and the +-axis
    // pairs the momentum balances, so the update conserves both to rounding.
    float rdl = 0.f, rF = 0.f, mdl[3] = {0.f, 0.f, 0.f}, mF[3] = {F[0], F[1], F[2]};
    bool bad = !(r > 0.f);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        float e = r, ed = r;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            e *= fac_of(fu[a], cc<D>(i, a));
            ed *= fac_of(fd[a], cc<D>(i, a));
        }
        float di = (e - wt<D>(i)) - fp[i];   // f^eq(u) - f = f^eq(u + du) - f'
        float Fi = ed - e;
        rdl += di;
        rF += Fi;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (cc<D>(i, a) != 0) {
                mdl[a] += (float)cc<D>(i, a) * di;
                mF[a] -= (float)cc<D>(i, a) * Fi;
            }
        dl[i] = di;
        fp[i] = (fp[i] + wt<D>(i)) + Fi;     // mirror state f' (Eq. mirror_state)
    }
    dl[0] = -rdl;
    fp[0] = (fp[0] + wt<D>(0)) - rF;
#pragma unroll
    for (int a = 0; a < D; ++a) {             // axis directions: i = 2a+1 (+e_a), 2a+2 (-e_a)
        dl[2 * a + 1] -= 0.5f * mdl[a];
        dl[2 * a + 2] += 0.5f * mdl[a];
        fp[2 * a + 1] += 0.5f * mF[a];
        fp[2 * a + 2] -= 0.5f * mF[a];
    }
    // x_i = D_i / f'_i (stored over dl)
    float xmax = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        bad |= !(fp[i] > 0.f);
        float xi = dl[i] * (1.0f / fp[i]);
        dl[i] = xi;
        xmax = fmaxf(xmax, fabsf(xi));
    }
    float al = 2.0f;
    if (bad) {
        atomicOr(status, STATUS_DIVERGED);
    } else if (xmax >= 1e-5f) {
        al = alpha_series<Q>(fp, dl);
        if (xmax > ALPHA_SERIES_MAX) {
            // positivity bound alpha_max = 1 / max(-x_i)
            float xneg = 0.f;
#pragma unroll
            for (int i = 0; i < Q; ++i) xneg = fmaxf(xneg, -dl[i]);
            const float amax = xneg > 0.f ? 1.0f / xneg : 3.0e38f;
            al = alpha_newton<Q>(fp, dl, amax, al);
        }
    }
    const float ab = al * local_beta(p, r, ph);

    // halfway bounce-back: bit i set when the neighbour x + c_i is solid (one
    // mask for the f and g stores).  FIRSTNB: only first-layer nodes have
    // solid neighbours, so the others skip the test (D3Q27, and the D2Q9
    // build for launches of more than one wave, which is issue-bound; the
    // one-wave D2Q9 build is latency-bound and measured faster without the
    // branch)
    unsigned solid_nb = 0;
    if (!FIRSTNB || (tc & TLB_FIRST)) {
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int m = (sx + cc<D>(i, 0)) + SX * ((sy + cc<D>(i, 1)) + SY * (sz + cc<D>(i, 2)));
            if (stype[m] & TLB_SOLID) solid_nb |= 1u << i;
        }
    }

    // f_new = f' + alpha beta D (Eq. ELBMequation); push streaming with halfway bounce-back
    {
        // direction i's array, advanced by N per direction
        float *fo = f_out;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float fn = (fp[i] - wt<D>(i)) + ab * (dl[i] * fp[i]);
            if (solid_nb & (1u << i))
                f_out[(long long)opp<D>(i) * p.N + n] = fn;
            else
                fo[nbr(cc<D>(i, 0), cc<D>(i, 1), cc<D>(i, 2))] = fn;
            fo += p.N;
        }
    }

    // ---- LBGK for g (Eq. CahnHilliardLBM) with g^eq(phi, v, mu_phi) ----
    float v2 = 0.f;
#pragma unroll
    for (int a = 0; a < D; ++a) v2 += v[a] * v[a];
    float gsum = 0.f, g0 = 0.f;
    // g^eq_i = w_i (3 Gamma mu_phi + 3 phi c.v + 4.5 phi (c.v)^2 - 1.5 phi v^2), factored in c.v
    const float gA = 3.0f * p.Gamma * mup - 1.5f * ph * v2, gB = 3.0f * ph, gC = 4.5f * ph;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        float gi;
        if ((ASYNC || FUSED) && sizeof(GT) == 4) {
            gi = stage[(Q + i) * NT + tid];
        } else if (FUSED || (ASYNC && (p.nx & 1) == 0)) {
            const __half *s16 = reinterpret_cast<const __half *>(&stage[(Q + 1) * NT]);
            gi = (i == 0) ? stage[Q * NT + tid] : __half2float(s16[(i - 1) * NT + tid]) * p.g_unscale;
        } else {
            gi = GIO<GT>::ld(g_in, i, n, p);
        }
        if (i == 0) { g0 = gi; continue; }
        float cv = 0.f;
#pragma unroll
        for (int a = 0; a < D; ++a) cv += (float)cc<D>(i, a) * v[a];
        float ge = wt<D>(i) * (gA + cv * (gB + gC * cv));
        gsum += ge;
        float gn = gi + (ge - gi) * p.inv_tau_g;
        if (solid_nb & (1u << i))
            GIO<GT>::st(g_out, opp<D>(i), n, gn, p);
        else if constexpr (sizeof(GT) == 4)
            ((float *)g_out + (long long)i * p.N)[nbr(cc<D>(i, 0), cc<D>(i, 1), cc<D>(i, 2))] = gn;
        else
            GIO<GT>::st(g_out, i, nbr(cc<D>(i, 0), cc<D>(i, 1), cc<D>(i, 2)), gn, p);
    }
    {
        float ge0 = ph - gsum;
        GIO<GT>::st(g_out, 0, n, g0 + (ge0 - g0) * p.inv_tau_g, p);
    }
}

template <int D, typename GT, int MODE>
__global__ void __launch_bounds__(256, D == 2 ? 4 : 2) step_kernel(DevParams p, const float *__restrict__ f_in, float *__restrict__ f_out,
                                                   const void *g_in, void *g_out, const float *__restrict__ rho,
                                                   const float *__restrict__ phi, const uint8_t *__restrict__ type,
                                                   unsigned *status, const float *__restrict__ u_init, AuxOut aux)
{
    int x0 = blockIdx.x * Tile<D>::X, y0 = blockIdx.y * Tile<D>::Y, z0 = blockIdx.z * Tile<D>::Z;
    step_tile<D, GT, MODE>(p, f_in, f_out, g_in, g_out, rho, phi, type, status, x0, y0, z0, u_init, aux);
}

// The stepping kernel of every lattice, alone or batched: one CTA per entry of
// a tile table (lattice index, tile origin).  A lattice advanced alone is a
// batch of one, so its results are bit-identical to the same lattice in a mix.
// MINB: resident CTAs per SM the registers are budgeted for.  D2Q9 comes in
// two builds with the same code (the register allocation alone differs):
// 3 CTAs/SM (80 registers, fewer spills) for launches that fit in one wave,
// 4 CTAs/SM (64 registers, more warps to hide latency) for larger ones.
template <int D, typename GT, int MINB>
__global__ void __launch_bounds__(256, MINB) step_batch_kernel(const BatchEntry *__restrict__ E, const int4 *__restrict__ tiles)
{
    __shared__ BatchEntry se;
    pdl_trigger();
    pdl_wait();
    const int4 t = tiles[blockIdx.x];
    static_assert(sizeof(BatchEntry) % 4 == 0 && sizeof(BatchEntry) / 4 <= 256, "entry copy");
    if (threadIdx.x < sizeof(BatchEntry) / 4)
        reinterpret_cast<int *>(&se)[threadIdx.x] = reinterpret_cast<const int *>(&E[t.x])[threadIdx.x];
    __syncthreads();
    AuxOut none = {};
    // D2Q9 tiles sum their own moments; D3Q27 tiles read those of the moments kernel
    step_tile<D, GT, MODE_STEP, D == 3, D == 2, (D == 3 || MINB == 4)>(se.p, se.f_in, se.f_out, se.g_in, se.g_out, se.rho, se.phi, se.type,
                                                se.status, t.y, t.z, t.w, nullptr, none, se.tm);
}

// ---------------------------------------------------------------------------
// fields: bare velocity u = sum f c / rho at fluid nodes
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) fields_kernel(DevParams p, const float *__restrict__ f, const float *__restrict__ rho,
                                                     const uint8_t *__restrict__ type, float *u)
{
    constexpr int Q = Lat<D>::Q;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < p.N; n += (long long)gridDim.x * blockDim.x) {
        float j[3] = {0.f, 0.f, 0.f};
        bool solid = type[n] & TLB_SOLID;
        if (!solid) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                float fi = f[(long long)i * p.N + n];
#pragma unroll
                for (int a = 0; a < D; ++a)
                    if (cc<D>(i, a) != 0) j[a] += (float)cc<D>(i, a) * fi;
            }
        }
        float ir = solid ? 0.f : 1.0f / rho[n];
#pragma unroll
        for (int a = 0; a < D; ++a) u[(long long)a * p.N + n] = j[a] * ir;
    }
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: per-block partial sums (fixed order), then one block.
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) diag_kernel(DevParams p, const float *__restrict__ f, const float *__restrict__ rho,
                                                   const float *__restrict__ phi, const uint8_t *__restrict__ type,
                                                   double *partials)
{
    constexpr int Q = Lat<D>::Q;
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < p.N; n += (long long)gridDim.x * blockDim.x) {
        if (type[n] & TLB_SOLID) continue;
        double r = rho[n], ph = phi[n];
        double C1 = (r - (double)p.rho_l) / ((double)p.rho_g - (double)p.rho_l);
        s[0] += r;
        s[1] += ph;
        s[2] += C1;
        s[3] += 0.5 * (1.0 + ph / (double)p.chi - C1);
        s[4] += 0.5 * (1.0 - ph / (double)p.chi - C1);
        double j[3] = {0, 0, 0};
        for (int i = 1; i < Q; ++i) {
            double fi = f[(long long)i * p.N + n];
            for (int a = 0; a < D; ++a) j[a] += cc<D>(i, a) * fi;
        }
        double j2 = 0;
        for (int a = 0; a < D; ++a) j2 += j[a] * j[a];
        s[5] += 0.5 * j2 / r;
    }
    __shared__ double red[6][8];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 6; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        partials[(long long)blockIdx.x * 6 + threadIdx.x] = v;
    }
}

template <int D>
__global__ void diag_final_kernel(const double *partials, int nblocks, double *out)
{
    if (threadIdx.x < 6) {
        double v = 0;
        for (int b = 0; b < nblocks; ++b) v += partials[(long long)b * 6 + threadIdx.x];
        out[threadIdx.x] = v;
    }
}

// populations <-> FP64 host-order buffers (dir 0: device -> double, 1: double -> device)
template <int D, typename GT>
__global__ void convert_kernel(DevParams p, float *f, void *g, double *fb, double *gb, int dir)
{
    constexpr int Q = Lat<D>::Q;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < p.N; n += (long long)gridDim.x * blockDim.x) {
        for (int i = 0; i < Q; ++i) {
            long long k = (long long)i * p.N + n;
            if (dir == 0) {
                fb[k] = (double)f[k] + (double)wt<D>(i);
                gb[k] = (double)GIO<GT>::ld(g, i, n, p);
            } else {
                f[k] = (float)(fb[k] - (double)wt<D>(i));
                GIO<GT>::st(g, i, n, (float)gb[k], p);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
inline int grid_for(long long N, int threads)
{
    long long b = (N + threads - 1) / threads;
    long long cap = 152LL * 16;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <int D>
int Launch<D>::Q() { return Lat<D>::Q; }

template <int D>
int Launch<D>::tile_dims(int a) { return a == 0 ? Tile<D>::X : a == 1 ? Tile<D>::Y : Tile<D>::Z; }

template <int D>
void Launch<D>::moments(const DevParams &p, const DevState &s, cudaStream_t st)
{
    if (p.g_fp16)
        moments_kernel<D, __half><<<grid_for(p.N, 256), 256, 0, st>>>(p, s.f[s.cur], s.g[s.cur], s.type, s.rho, s.phi);
    else
        moments_kernel<D, float><<<grid_for(p.N, 256), 256, 0, st>>>(p, s.f[s.cur], s.g[s.cur], s.type, s.rho, s.phi);
}

template <int D>
void Launch<D>::ghosts(const DevParams &p, const DevState &s, cudaStream_t st)
{
    if (s.nghost > 0)
        ghost_kernel<D><<<(s.nghost + 127) / 128, 128, 0, st>>>(p, s.type, s.rho, s.phi, s.ghosts, s.nghost);
}

template <int D>
void Launch<D>::step(const DevParams &p, const DevState &s, int mode, const float *u_init, AuxOut aux, cudaStream_t st)
{
    dim3 grid((p.nx + Tile<D>::X - 1) / Tile<D>::X, (p.ny + Tile<D>::Y - 1) / Tile<D>::Y,
              (p.nz + Tile<D>::Z - 1) / Tile<D>::Z);
    dim3 block(Tile<D>::X * Tile<D>::Y * Tile<D>::Z);
    int cur = s.cur, nxt = 1 - s.cur;
#define TLB_LAUNCH_STEP(GT)                                                                                          \
    do {                                                                                                             \
        if (mode == MODE_STEP)                                                                                       \
            step_kernel<D, GT, MODE_STEP><<<grid, block, 0, st>>>(p, s.f[cur], s.f[nxt], s.g[cur], s.g[nxt], s.rho,   \
                                                                   s.phi, s.type, s.status, nullptr, aux);           \
        else if (mode == MODE_INIT)                                                                                  \
            step_kernel<D, GT, MODE_INIT><<<grid, block, 0, st>>>(p, s.f[cur], s.f[cur], s.g[cur], s.g[cur], s.rho,   \
                                                                   s.phi, s.type, s.status, u_init, aux);            \
        else                                                                                                         \
            step_kernel<D, GT, MODE_AUX><<<grid, block, 0, st>>>(p, s.f[cur], s.f[cur], s.g[cur], s.g[cur], s.rho,    \
                                                                  s.phi, s.type, s.status, nullptr, aux);            \
    } while (0)
    if (p.g_fp16) TLB_LAUNCH_STEP(__half);
    else TLB_LAUNCH_STEP(float);
#undef TLB_LAUNCH_STEP
}

template <int D>
void Launch<D>::fields(const DevParams &p, const DevState &s, float *u_out, cudaStream_t st)
{
    fields_kernel<D><<<grid_for(p.N, 256), 256, 0, st>>>(p, s.f[s.cur], s.rho, s.type, u_out);
}

template <int D>
int Launch<D>::diag_blocks(const DevParams &p) { return grid_for(p.N, 256) < 1024 ? grid_for(p.N, 256) : 1024; }

template <int D>
void Launch<D>::diagnostics(const DevParams &p, const DevState &s, double *partials, int nblocks, double *out,
                            cudaStream_t st)
{
    diag_kernel<D><<<nblocks, 256, 0, st>>>(p, s.f[s.cur], s.rho, s.phi, s.type, partials);
    diag_final_kernel<D><<<1, 32, 0, st>>>(partials, nblocks, out);
}

template <int D>
void Launch<D>::convert_pop(const DevParams &p, const DevState &s, int dir, double *fbuf, double *gbuf, cudaStream_t st)
{
    if (p.g_fp16)
        convert_kernel<D, __half><<<grid_for(p.N, 256), 256, 0, st>>>(p, s.f[s.cur], s.g[s.cur], fbuf, gbuf, dir);
    else
        convert_kernel<D, float><<<grid_for(p.N, 256), 256, 0, st>>>(p, s.f[s.cur], s.g[s.cur], fbuf, gbuf, dir);
}

// launch with programmatic stream serialization (the kernel's griddepcontrol.wait
// orders it after its predecessor's memory operations)
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int D>
unsigned Launch<D>::bounds_errors()
{
#ifdef TLB_BOUNDS_CHECK
    unsigned v = 0, zero = 0;
    cudaMemcpyFromSymbol(&v, g_bounds_error, sizeof(v));
    cudaMemcpyToSymbol(g_bounds_error, &zero, sizeof(zero));
    return v;
#else
    return 0;
#endif
}

template <int D>
void Launch<D>::moments_batch(const BatchEntry *entries, const int4 *tiles, int ntiles, int g_fp16, cudaStream_t st)
{
    if (ntiles <= 0) return;
    const int nt = Tile<D>::X * Tile<D>::Y * Tile<D>::Z;
    if (g_fp16) launch_pdl(moments_batch_kernel<D, __half>, ntiles, nt, 0, st, entries, tiles);
    else launch_pdl(moments_batch_kernel<D, float>, ntiles, nt, 0, st, entries, tiles);
}

template <int D, typename GT>
static void launch_step_batch(const BatchEntry *entries, const int4 *tiles, int ntiles, cudaStream_t st, int variant)
{
    constexpr int bytes = stage_bytes<D, GT>();
    constexpr int nt = Tile<D>::X * Tile<D>::Y * Tile<D>::Z;
    // once per process, on the first launch (thread-safe static initialisation):
    // the dynamic shared-memory opt-ins, and the SM count of the device that
    // runs the library (D2Q9: the one-wave bound)
    static const int nsm = [] {
        constexpr int b = stage_bytes<D, GT>();
        if constexpr (D == 2) {
            cudaFuncSetAttribute(step_batch_kernel<D, GT, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
            cudaFuncSetAttribute(step_batch_kernel<D, GT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        } else {
            cudaFuncSetAttribute(step_batch_kernel<D, GT, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        }
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n;
    }();
    if constexpr (D == 2) {
        const bool four = variant < 0 ? ntiles > 3 * nsm : variant == 1;
        if (four) launch_pdl(step_batch_kernel<D, GT, 4>, ntiles, nt, (size_t)bytes, st, entries, tiles);
        else launch_pdl(step_batch_kernel<D, GT, 3>, ntiles, nt, (size_t)bytes, st, entries, tiles);
    } else {
        launch_pdl(step_batch_kernel<D, GT, 2>, ntiles, nt, (size_t)bytes, st, entries, tiles);
    }
}

template <int D>
void Launch<D>::step_batch(const BatchEntry *entries, const int4 *tiles, int ntiles, int g_fp16, cudaStream_t st,
                           int variant)
{
    if (ntiles <= 0) return;
    if (g_fp16) launch_step_batch<D, __half>(entries, tiles, ntiles, st, variant);
    else launch_step_batch<D, float>(entries, tiles, ntiles, st, variant);
}


}  // namespace tlb
