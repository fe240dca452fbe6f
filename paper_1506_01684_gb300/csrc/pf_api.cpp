// pf_api.cpp -- host runtime behind the C ABI of include/pf.h: device buffers, the per-step
// launch sequence of Algorithm 1 (phi-sweep, mu-sweep, FP64 reductions, window), the
// Voronoi seeds, and the field/diagnostic transfers.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pf_internal.h"

using namespace pf;

// Launch shape of the fused step with the lean kernel.  The general planes' sweeps (latency-bound) run
// on a second stream beside the lean kernel (HBM-bound), so that the two kernels fill each other's
// tails (PF_CONCURRENT 1; 0: the sweeps after the lean kernel on the simulation's stream): 0.273
// against 0.293 ms a step on 256x256x1024 FP32.  The sweeps are launched first and with the device's
// highest priority; neither the order nor the priority changed the time measurably.  Persistent
// general CTAs per SM: two (they take all of an SM's registers while they run; one makes the sweeps
// 1.5x slower and the step slower than the serial form).
#ifndef PF_CONCURRENT
#define PF_CONCURRENT 1
#endif
#ifndef PF_GENERAL_CTAS_PER_SM
#define PF_GENERAL_CTAS_PER_SM 2
#endif


#ifndef PF_LEAN_PLANES
#define PF_LEAN_PLANES 64  // at most planes per lean CTA (the kernels' limit, PF_LEAN_PLANES in pf_kernels.cuh)
#endif
// the step's kernels launched with programmatic dependent launch (1), or plainly (0)
#ifndef PF_PDL
#define PF_PDL 1
#endif

// the general planes as the two sweeps of Algorithm 1 (1) or as the fused tile (0)
#ifndef PF_GENERAL_SWEEPS
#define PF_GENERAL_SWEEPS 1
#endif


// ------------------------------------------------------------------------------------------
// allocator hooks
// ------------------------------------------------------------------------------------------
namespace {
std::mutex g_alloc_mu;
pf_alloc_fn g_alloc = nullptr;
pf_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    pf_free_fn fr = nullptr;  // hook that allocated it (nullptr: cudaMalloc)
    void *ctx = nullptr;
};

int dev_alloc(DevBuf &b, size_t bytes, cudaStream_t s)
{
    pf_alloc_fn a;
    pf_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
        f = g_free;
        ctx = g_alloc_ctx;
    }
    b.bytes = bytes;
    if (a) {
        b.p = a(bytes, (void *)s, ctx);
        b.fr = f;
        b.ctx = ctx;
        return b.p ? PF_OK : PF_E_NOMEM;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return e == cudaErrorMemoryAllocation ? PF_E_NOMEM : PF_E_CUDA;
    }
    return PF_OK;
}

void dev_free(DevBuf &b, cudaStream_t s)
{
    if (!b.p) return;
    if (b.fr)
        b.fr(b.p, b.bytes, (void *)s, b.ctx);
    else
        cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// splitmix64 (Steele, Lea and Flood 2014): golden-ratio increment, then the variant-13 mixer.
uint64_t splitmix64_next(uint64_t &state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
double unit53(uint64_t &state) { return (double)(splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

// ------------------------------------------------------------------------------------------
// simulation object
// ------------------------------------------------------------------------------------------
struct pf_sim {
    int nx, ny, nz;
    pf_params p;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the general planes' sweeps beside the lean kernel: a stream of the highest priority, so that
    // their persistent CTAs are placed before the lean kernel's; events for the fork and the join
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    Geometry geo;          // unfused sweeps
    Geometry geo_fused;    // fused step (longer z chunks: its prologue recomputes two planes)
    int variant = PF_VARIANT_AUTO;
    // PF_VARIANT_AUTO's measured choice for the current run: -1 not yet measured, 0 the default rule's
    // path, 1 the two whole-domain sweeps (faster on this domain's composition)
    int auto_choice = -1;
    DevBuf phi[2], mu[2];  // AoS fields of the stencil precision
    DevBuf philo[2], mulo[2];  // low words of the compensated FP32 state (PF_FP32_COMP only)
    // liquid maps of the two field buffers (one byte per storage plane and fused-step tile: 1 when
    // the tile's cells of that plane are exactly pure liquid); written by every fused step for its
    // new field, rebuilt by the classify kernel where tmap_ok says the map is stale
    DevBuf tmap[2];
    bool tmap_ok[2] = {false, false};
    // TMA tensor maps of the two mu buffers for the lean kernel (the fused step's pure-liquid
    // planes); lean_ok when both could be encoded (FP32 rows must be 16-byte multiples: nx even)
    LeanMaps mu_map[2];
    DevBuf lean_stats;  // LeanStats
    DevBuf splits;      // int2 per (tile, chunk) of the fused grid: the lean / general split
    DevBuf glist;       // int per (tile, chunk): the items with general planes
    DevBuf subparts;    // Partial per work unit of the general planes (kMaxUnits per item)
    DevBuf subcnt;      // unsigned per (tile, chunk): units of the item finished in this step
    int general_ctas = 0;  // persistent CTAs of the general kernel
    int gphi_ctas = 0, gmu_ctas = 0;  // persistent CTAs of the general planes' two sweeps
    bool lean_ok = false;
    int lean_nsub = 1;  // lean CTAs per z chunk of the fused grid
    DevBuf state;          // DevState
    DevBuf parts;          // Partial[geo.nparts()]
    DevBuf tab;            // PlaneT<R>[2 nz]
    DevBuf seeds;          // Voronoi seeds
    DevBuf red;            // nz x 8 FP64 plane sums
    int cur = 0;           // index of the source buffers
    int latched = PF_OK;
    // per-kernel timers
    bool prof = false;
    struct Rec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    // a captured graph of two steps (buffers 0 -> 1 -> 0), rebuilt when the variant changes
    cudaGraphExec_t graph = nullptr;
    int graph_variant = -1;
    long long direct_steps = 0;
    bool use_graphs = true;
    int last_nparts = 0;  // partial sums written by the last step's kernels
    int last_kind = -1;   // 0: two sweeps, 1: fused kernel alone, 2: fused kernel + lean kernel
    bool test_withhold = false;  // test hook: the lean kernel's producer issues no copies
    // a slab of a decomposed domain (pf_split): local row j is global row (j + gy0) mod gny; own rows
    // [red_j0, red_j1) (gny = 0: not a slab)
    int gy0 = 0, gny = 0, red_j0 = 0, red_j1 = 0;
    size_t ncell() const { return (size_t)nx * ny * nz; }
    size_t wbytes() const { return p.precision == PF_FP64 ? 8 : 4; }
    bool comp() const { return p.precision == PF_FP32_COMP; }
    void *lo_phi(int b) const { return comp() ? philo[b].p : nullptr; }
    void *lo_mu(int b) const { return comp() ? mulo[b].p : nullptr; }
};

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor maps of one mu buffer for the lean kernel (LeanMaps): 3D (2 nx words, ny rows, nz storage
// planes), boxes of (TX + 4) cells x (TY + 2) rows (the tile with its halo), 2 cells x TY rows (the
// periodic x images) and (TX + 4) cells x 1 row (the periodic y images); zero fill outside.  False when
// the layout does not allow them (rows must be 16-byte multiples).
static bool encode_lean_maps(LeanMaps *m, void *base, int nx, int ny, int nz, size_t w, int tx, int ty)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base || ((uintptr_t)base & 15) || ((size_t)2 * nx * w) % 16 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)2 * nx * w, (cuuint64_t)2 * nx * ny * w};
    const cuuint32_t es[3] = {1, 1, 1};
    const cuuint32_t boxes[3][3] = {{(cuuint32_t)(2 * (tx + 4)), (cuuint32_t)(ty + 2), 1},
                                    {4, (cuuint32_t)ty, 1},
                                    {(cuuint32_t)(2 * (tx + 4)), 1, 1}};
    CUtensorMap *out[3] = {&m->box, &m->ximg, &m->yimg};
    for (int k = 0; k < 3; k++) {
        const CUresult r = enc(out[k], w == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                               base, dims, strides, boxes[k], es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

namespace pf {
Geometry make_geometry(int nx, int ny, int nz, int zchunk_hint)
{
    Geometry g;
    g.tx = 32;
    g.ty = 8;
    g.gx = (nx + g.tx - 1) / g.tx;
    g.gy = (ny + g.ty - 1) / g.ty;
    int zc = zchunk_hint;
    if (zc <= 0) {
        // aim at >= 16 CTAs per SM of 152 SMs; 8..64 planes per CTA (each chunk re-reads 2 planes)
        const long tiles = (long)g.gx * g.gy;
        long chunks = (152L * 16 + tiles - 1) / tiles;
        zc = (int)((nz + chunks - 1) / chunks);
        zc = std::max(8, std::min(64, zc));
    }
    zc = std::max(1, std::min(zc, nz));
    g.zchunk = zc;
    g.gz = (nz + zc - 1) / zc;
    return g;
}
}  // namespace pf

static bool tau_pairs(const pf_params &p);

template <typename R>
static KParams<R> make_kparams(const pf_sim *s)
{
    const pf_params &p = s->p;
    KParams<R> k;
    memset(&k, 0, sizeof k);
    k.nx = s->nx;
    k.ny = s->ny;
    k.nz = s->nz;
    k.zchunk = s->geo.zchunk;
    k.window = p.window_trigger_z > 0.0 ? 1 : 0;
    k.tgx = s->geo_fused.gx;
    k.tgy = s->geo_fused.gy;
    k.test_flags = s->test_withhold ? 1 : 0;
    k.gy0 = s->gy0;
    k.gny = s->gny;
    k.red_j0 = s->red_j0;
    k.red_j1 = s->red_j1;
    k.dx = (R)p.dx;
    k.inv_dx = (R)(1.0 / p.dx);
    k.inv_2dx = (R)(1.0 / (2.0 * p.dx));
    k.inv_4dx = (R)(1.0 / (4.0 * p.dx));
    k.eps = (R)p.eps;
    k.inv_eps = (R)(1.0 / p.eps);
    k.c_phi = (R)(p.dt / (p.tau * p.eps));
    k.dt = (R)p.dt;
    k.inv_dt = (R)(1.0 / p.dt);
    for (int q = 0; q < 6; q++) k.gamma2[q] = (R)p.gamma2[q];
    for (int q = 0; q < 4; q++) k.gamma3[q] = (R)p.gamma3[q];
    for (int a = 0; a < 4; a++) {
        k.inv2A[a] = (R)(1.0 / (2.0 * p.A[a]));
        k.inv4A[a] = (R)(1.0 / (4.0 * p.A[a]));
        k.DinvA[a] = (R)(p.D[a] / (2.0 * p.A[a]));
        k.kT[a][0] = (R)p.kT[a][0];
        k.kT[a][1] = (R)p.kT[a][1];
        k.cE[a][0] = p.cE[a][0];
        k.cE[a][1] = p.cE[a][1];
        k.kT64[a][0] = p.kT[a][0];
        k.kT64[a][1] = p.kT[a][1];
        k.s64[a] = p.s[a];
        k.A64[a] = p.A[a];
    }
    // K_a = (1/2) A_a^{-1} in FP64 (the identity form when Am[a] is not set)
    k.gen = 0;
    for (int a = 0; a < 4; a++) {
        double K11, K12, K22;
        if (p.Am[a][0] > 0.0) {
            k.gen = 1;
            const double a11 = p.Am[a][0], a12 = p.Am[a][1], a22 = p.Am[a][2];
            const double det = a11 * a22 - a12 * a12;
            K11 = 0.5 * a22 / det;
            K12 = -0.5 * a12 / det;
            K22 = 0.5 * a11 / det;
        } else {
            K11 = K22 = 1.0 / (2.0 * p.A[a]);
            K12 = 0.0;
        }
        const double Kd[3] = {K11, K12, K22};
        for (int e = 0; e < 3; e++) {
            k.K64[a][e] = Kd[e];
            k.K[a][e] = (R)Kd[e];
            k.DK[a][e] = (R)(p.D[a] * Kd[e]);
        }
        k.psiK[a][0] = (R)(0.5 * K11);
        k.psiK[a][1] = (R)K12;
        k.psiK[a][2] = (R)(0.5 * K22);
    }
    k.gen_tau = tau_pairs(p) ? 1 : 0;
    for (int q = 0; q < 6; q++) k.tau_ab[q] = (R)(k.gen_tau ? p.tau_ab[q] : p.tau);
    k.dt_eps = (R)(p.dt / p.eps);
    {
        // pure liquid: chi = K_l, M = D_l K_l, so chi^{-1} M = D_l and the source of the
        // temperature drift is -K_l^{-1} kT_l dT
        const double K11 = k.K64[3][0], K12 = k.K64[3][1], K22 = k.K64[3][2];
        const double det = K11 * K22 - K12 * K12, dT = -p.G * p.v * p.dt;
        const double s0 = p.kT[3][0] * dT, s1 = p.kT[3][1] * dT;
        k.liqC1 = (R)(p.dt * p.D[3] / (p.dx * p.dx));
        k.liqC0[0] = (R)(-(K22 * s0 - K12 * s1) / det);
        k.liqC0[1] = (R)(-(K11 * s1 - K12 * s0) / det);
    }
    const double pi = 3.14159265358979323846;
    k.at_pref = (R)(pi * p.eps / 4.0);
    k.grad_thr = (R)(1e-20 / (p.dx * p.dx));
    k.obst = (R)(16.0 / (pi * pi));
    k.dTstep = (R)(-p.G * p.v * p.dt);
    k.T0 = p.T0;
    k.G = p.G;
    k.v = p.v;
    k.TE = p.TE;
    k.dx64 = p.dx;
    k.dt64 = p.dt;
    k.eps64 = p.eps;
    k.window_trigger_z = p.window_trigger_z;
    return k;
}

// ------------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------------
static double default_dt(const pf_params &p, int nz);
static int check_params(const pf_params *p);

namespace pf {
// Kernel parameters for a grid without a pf_sim (used by the allocation-free entry point).
template <typename R>
KParams<R> kparams_for(const pf_params &p, int nx, int ny, int nz, const Geometry &g)
{
    pf_sim tmp;
    tmp.nx = nx;
    tmp.ny = ny;
    tmp.nz = nz;
    tmp.p = p;
    tmp.geo = g;
    tmp.geo_fused = g;
    return make_kparams<R>(&tmp);
}
template KParams<float> kparams_for<float>(const pf_params &, int, int, int, const Geometry &);
template KParams<double> kparams_for<double>(const pf_params &, int, int, int, const Geometry &);
double resolved_dt(const pf_params &p, int nz) { return p.dt > 0.0 ? p.dt : default_dt(p, nz); }
int validate_params(const pf_params *p) { return check_params(p); }
}  // namespace pf

static int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return PF_OK;
    if (e == cudaErrorMemoryAllocation) return PF_E_NOMEM;
    return PF_E_CUDA;
}

static int latch(pf_sim *s, int st)
{
    if (st != PF_OK && s->latched == PF_OK) s->latched = st;
    return st;
}

static bool tau_pairs(const pf_params &p)
{
    for (int q = 0; q < 6; q++)
        if (p.tau_ab[q] > 0.0) return true;
    return false;
}

static double default_dt(const pf_params &p, int nz)
{
    double gmax = 0.0, dmax = 0.0, tmin = p.tau;
    if (tau_pairs(p))
        for (int q = 0; q < 6; q++) tmin = p.tau_ab[q] < tmin ? p.tau_ab[q] : tmin;
    for (int i = 0; i < 6; i++) gmax = p.gamma2[i] > gmax ? p.gamma2[i] : gmax;
    for (int a = 0; a < 4; a++) dmax = p.D[a] > dmax ? p.D[a] : dmax;
    const double Ttop = p.T0 + p.G * (double)(nz - 1) * p.dx;
    const double Tmax = p.T0 > Ttop ? p.T0 : Ttop;
    const double lim_phi = tmin * p.dx * p.dx / (12.0 * gmax * Tmax);
    const double lim_mu = dmax > 0.0 ? p.dx * p.dx / (6.0 * dmax) : lim_phi;
    return 0.5 * (lim_phi < lim_mu ? lim_phi : lim_mu);
}

static int check_params(const pf_params *p)
{
    if (!p || p->version != PF_PARAMS_VERSION) return PF_E_INVAL;
    if (p->precision != PF_FP64 && p->precision != PF_FP32 && p->precision != PF_FP32_COMP) return PF_E_INVAL;
    if (!(p->dx > 0) || !(p->eps > 0) || !(p->tau > 0)) return PF_E_INVAL;
    for (int a = 0; a < 4; a++) {
        if (!(p->A[a] > 0) || p->D[a] < 0) return PF_E_INVAL;
        const double a11 = p->Am[a][0], a12 = p->Am[a][1], a22 = p->Am[a][2];
        if (a11 > 0 && !(a22 > 0 && a11 * a22 - a12 * a12 > 0 && isfinite(a12))) return PF_E_INVAL;
    }
    if (tau_pairs(*p))
        for (int q = 0; q < 6; q++)
            if (!(p->tau_ab[q] > 0) || !isfinite(p->tau_ab[q])) return PF_E_INVAL;
    double gmax = 0;
    for (int i = 0; i < 6; i++) gmax = std::max(gmax, p->gamma2[i]);
    if (!(gmax > 0)) return PF_E_INVAL;
    if (p->seed_layers < 0 || p->n_grains < 0) return PF_E_INVAL;
    if (!isfinite(p->T0) || !isfinite(p->G) || !isfinite(p->v) || !isfinite(p->TE)) return PF_E_INVAL;
    return PF_OK;
}

// ------------------------------------------------------------------------------------------
// precision-dispatched bodies
// ------------------------------------------------------------------------------------------
static cudaEvent_t pool_event(pf_sim *s)
{
    if (!s->pool.empty()) {
        cudaEvent_t e = s->pool.back();
        s->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch f() on stream st (default: the sim's stream), bracketed by timing events when profiling
// is on.
template <typename F>
static cudaError_t timed(pf_sim *s, int cls, F &&f, cudaStream_t st = nullptr)
{
    if (!st) st = s->stream;
    if (!s->prof) return f();
    cudaEvent_t a = pool_event(s), b = pool_event(s);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = f();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    s->recs.push_back({cls, a, b});
    return e;
}

// AUTO: the lean path (plan, lean kernel, general planes' sweeps) wherever the lean kernel's tensor maps
// exist, in every precision (measured on 256x256x1024 after 2000 steps: FP64 11.5 against 2.1 GLUP/s with
// the two whole-domain sweeps, compensated FP32 130 against 22); without them the fused tile in FP32
// and the two sweeps otherwise.  A fixed rule, not a timing: a run resumed from a checkpoint takes the
// same kernels as the uninterrupted run.
// The step's path under the default rule: the lean path wherever it can run (FP32 rows of 16-byte
// multiples, every precision), else in FP32 the fused tile, else the two whole-domain sweeps.
static bool rule_fused(const pf_sim *s)
{
    // the compensated state has a lean path (lean kernel and general planes' sweeps with the low
    // words), but no fused tile: without the lean path it runs on the two sweeps
    if (s->comp()) return s->lean_ok;
    return s->lean_ok || s->p.precision == PF_FP32;
}
static bool use_fused(const pf_sim *s)
{
    if (s->variant == PF_VARIANT_UNFUSED) return false;
    if (s->variant == PF_VARIANT_FUSED) return s->comp() ? s->lean_ok : true;
    // AUTO: the rule's path unless a measurement on this run's state found the two sweeps faster
    return s->auto_choice != 1 && rule_fused(s);
}

// The fused step trusts the liquid maps of both field buffers: the source's to find the
// pure-liquid planes, the destination's (which describes the field two steps back) to skip the
// phi stores of planes that stay pure liquid.  Rebuild whichever map is stale.
// A rebuilt liquid map (the fields changed outside the lean path) makes the device-side plan stale: the
// next plan kernel lists the items afresh.
static cudaError_t invalidate_plan(pf_sim *s, cudaStream_t stream)
{
    unsigned char *ls = (unsigned char *)s->lean_stats.p;
    cudaError_t e = cudaMemsetAsync(ls + offsetof(LeanStats, plan_valid), 0, sizeof(int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ls + offsetof(LeanStats, gcount), 0, sizeof(unsigned), stream);
    return e;
}

template <typename R>
static cudaError_t ensure_maps(pf_sim *s, cudaStream_t stream)
{
    const KParams<R> kp = make_kparams<R>(s);
    for (int b = 0; b < 2; b++) {
        if (s->tmap_ok[b]) continue;
        cudaError_t e = launch_classify<R>(kp, (const DevState *)s->state.p, s->phi[b].p,
                                           (unsigned char *)s->tmap[b].p, stream, s->lo_phi(b));
        if (e == cudaSuccess) e = invalidate_plan(s, stream);
        if (e != cudaSuccess) return e;
        s->tmap_ok[b] = true;
    }
    return cudaSuccess;
}

// The second stream and the fork / join events of the general planes' sweeps beside the lean kernel,
// made on the first step that takes the lean path (not while the simulation's stream is being
// captured: such a step runs the sweeps after the lean kernel).
static void ensure_aux(pf_sim *s)
{
    if (!PF_CONCURRENT || s->aux) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return;
    }
    int lo = 0, hi = 0;
    cudaStream_t x = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&x, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming);
    if (e != cudaSuccess) {  // the serial form needs none of them
        cudaGetLastError();
        if (x) cudaStreamDestroy(x);
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        return;
    }
    s->aux = x;
    s->ev_fork = a;
    s->ev_join = b;
}

template <typename R>
static int do_step_direct(pf_sim *s, int n)
{
    const bool fused = use_fused(s);
    KParams<R> kp = make_kparams<R>(s);
    if (fused) kp.zchunk = s->geo_fused.zchunk;
    DevState *st = (DevState *)s->state.p;
    PlaneT<R> *tab = (PlaneT<R> *)s->tab.p;
    Partial *parts = (Partial *)s->parts.p;
    const bool lean = fused && s->lean_ok;
    if (lean) ensure_aux(s);
    const int np_fused = s->geo_fused.nparts();
    const int nparts = fused ? np_fused : s->geo.nparts();
    s->last_nparts = nparts;
    s->last_kind = fused ? (lean ? 2 : 1) : 0;
    for (int q = 0; q < n; q++) {
        const int a = s->cur, b = 1 - s->cur;
        cudaError_t e;
        if (fused) {
            e = ensure_maps<R>(s, s->stream);
            const unsigned char *tin = (const unsigned char *)s->tmap[a].p;
            unsigned char *tout = (unsigned char *)s->tmap[b].p;
            LeanStats *ls = (LeanStats *)s->lean_stats.p;
            if (!lean) {
                if (e == cudaSuccess)
                    e = timed(s, PF_K_FUSED, [&] {
                        return launch_fused_step<R>(kp, s->geo_fused, s->phi[a].p, s->mu[a].p, s->phi[b].p,
                                                    s->mu[b].p, st, tab, parts, s->stream, tin, tout, true);
                    });
            } else {
                // plan the step (splits, list of items with general planes), the lean planes, then the
                // general planes' two sweeps.  The general planes touch other planes, map entries and
                // partials than the lean kernel, so with programmatic dependent launch the phi-sweep's
                // CTAs start as the lean kernel's last CTAs retire
                const bool pdl = PF_PDL != 0;
                auto general = [&]() -> cudaError_t {
                    if (PF_GENERAL_SWEEPS)
                        return timed(s, PF_K_GENERAL, [&] {
                            return launch_general_sweeps<R>(kp, s->phi[a].p, s->mu[a].p, s->phi[b].p, s->mu[b].p, st,
                                                            tab, parts, tin, tout, (const int2 *)s->splits.p,
                                                            (const int *)s->glist.p, ls, s->gphi_ctas, s->gmu_ctas,
                                                            s->stream, (Partial *)s->subparts.p,
                                                            (unsigned *)s->subcnt.p, pdl, true, s->lo_phi(a),
                                                            s->lo_phi(b), s->lo_mu(a), s->lo_mu(b));
                        });
                    return timed(s, PF_K_FUSED, [&] {
                        return launch_general_step<R>(kp, s->phi[a].p, s->mu[a].p, s->phi[b].p, s->mu[b].p, st, tab,
                                                      parts, tin, tout, (const int2 *)s->splits.p,
                                                      (const int *)s->glist.p, ls, s->general_ctas, s->stream);
                    });
                };
                auto leanp = [&]() -> cudaError_t {
                    return timed(s, PF_K_LEAN, [&] {
                        return launch_lean_step<R>(kp, s->geo_fused, s->lean_nsub, &s->mu_map[a], s->mu[a].p,
                                                   s->phi[b].p, s->mu[b].p, st, ls, s->stream, tin, tout,
                                                   (const int2 *)s->splits.p, pdl, s->lo_mu(a), s->lo_phi(b),
                                                   s->lo_mu(b));
                    });
                };
                if (e == cudaSuccess)
                    e = timed(s, PF_K_PLAN, [&] {
                        return launch_plan<R>(kp, s->geo_fused, st, tin, (int2 *)s->splits.p, (int *)s->glist.p, ls,
                                              parts, s->stream, pdl);
                    });
                if (s->aux && !s->prof && PF_GENERAL_SWEEPS) {
                    // the general planes' sweeps (latency-bound) beside the lean kernel (HBM-bound): both
                    // start once the plan is done; the general sweeps go first, on the stream of the
                    // highest priority, and finalize waits for both
                    if (e == cudaSuccess) e = cudaEventRecord(s->ev_fork, s->stream);
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->aux, s->ev_fork, 0);
                    if (e == cudaSuccess)
                        e = launch_general_sweeps<R>(kp, s->phi[a].p, s->mu[a].p, s->phi[b].p, s->mu[b].p, st, tab,
                                                     parts, tin, tout, (const int2 *)s->splits.p,
                                                     (const int *)s->glist.p, ls, s->gphi_ctas, s->gmu_ctas, s->aux,
                                                     (Partial *)s->subparts.p, (unsigned *)s->subcnt.p, false, false,
                                                     s->lo_phi(a), s->lo_phi(b), s->lo_mu(a), s->lo_mu(b), true);
                    if (e == cudaSuccess) e = cudaEventRecord(s->ev_join, s->aux);
                    if (e == cudaSuccess) e = leanp();
                    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->ev_join, 0);
                } else {
                    if (e == cudaSuccess) e = leanp();
                    if (e == cudaSuccess) e = general();
                }
            }
        } else if (s->comp()) {
            const KParams<float> &kf = reinterpret_cast<const KParams<float> &>(kp);
            const PlaneT<float> *tf = reinterpret_cast<const PlaneT<float> *>(tab);
            e = timed(s, PF_K_PHI, [&] {
                return launch_phi_sweep_comp(kf, s->geo, s->phi[a].p, s->philo[a].p, s->mu[a].p, s->phi[b].p,
                                             s->philo[b].p, st, tf, s->stream);
            });
            if (e == cudaSuccess)
                e = timed(s, PF_K_MU, [&] {
                    return launch_mu_sweep_comp(kf, s->geo, s->phi[a].p, s->phi[b].p, s->mu[a].p, s->mulo[a].p,
                                                s->mu[b].p, s->mulo[b].p, st, tf, parts, s->stream);
                });
        } else {
            e = timed(s, PF_K_PHI, [&] {
                return launch_phi_sweep<R>(kp, s->geo, s->phi[a].p, s->mu[a].p, s->phi[b].p, st, tab, s->stream);
            });
            if (e == cudaSuccess)
                e = timed(s, PF_K_MU, [&] {
                    return launch_mu_sweep<R>(kp, s->geo, s->phi[a].p, s->phi[b].p, s->mu[a].p, s->mu[b].p, st, tab,
                                              parts, s->stream);
                });
        }
        if (e == cudaSuccess)
            e = timed(s, PF_K_FINALIZE, [&] {
                return launch_finalize<R>(kp, st, parts, nparts, s->stream,
                                          lean ? (LeanStats *)s->lean_stats.p : nullptr,
                                          lean && PF_PDL && !(s->aux && !s->prof));
            });
        if (e == cudaSuccess)
            e = timed(s, PF_K_POST, [&] {
                return launch_post<R>(kp, st, s->phi[b].p, s->mu[b].p, tab, s->stream, s->lo_phi(b), s->lo_mu(b),
                                      fused ? (unsigned char *)s->tmap[b].p : nullptr, lean && PF_PDL);
            });
        if (e != cudaSuccess) return latch(s, cuda_status(e));
        s->tmap_ok[b] = fused;
        s->cur = b;
    }
    return PF_OK;
}

// pf_step's driver: direct launches while profiling (every kernel bracketed by events), for the
// first steps, for short calls and inside a caller's own stream capture; otherwise replays of a
// captured two-step graph (launch overhead of the four kernels per step paid once).
// PF_VARIANT_AUTO's choice for a run, made on the first step after its state was set (pf_init,
// pf_write_fields*, a checkpoint without a stored choice) from the state itself, so that two runs from
// the same state choose alike.  The lean path moves 16 bytes a pure-liquid cell and runs the general
// planes' persistent sweeps beside the lean kernel; the two whole-domain sweeps are grid launches.
// The measure is the fraction f of the (tile, plane) entries of the current field's liquid map that
// are exactly pure liquid; the lean path is kept when f reaches a threshold that depends on the
// domain's size, set from the region study (the paper's liquid, solid and interface blocks at 60^3,
// 128^3 and 256^3, FP32, GB300): below 2^20 cells the lean path was as fast or faster on every block
// (0: always kept); up to 2^23 cells the sweeps were 17-48 % faster on the solid and interface blocks
// (f <= 0.48) and the lean path 4.3x faster on pure liquid (0.6); above, the lean path was 7 % faster
// on the interface block (f ~ 0.48) and the sweeps 14 % on the solid one (0.45).
constexpr double kAutoLeanFractionMid = 0.6, kAutoLeanFractionLarge = 0.45;
constexpr size_t kAutoSmallCells = (size_t)1 << 20, kAutoLargeCells = (size_t)1 << 23;

template <typename R>
static int auto_choose(pf_sim *s)
{
    s->auto_choice = 0;
    if (!rule_fused(s) || !s->lean_ok) return PF_OK;  // the lean path cannot run: the rule stands
    cudaError_t e = ensure_maps<R>(s, s->stream);
    const size_t nmap = s->tmap[0].bytes;
    std::vector<unsigned char> h(nmap);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), s->tmap[s->cur].p, nmap, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return latch(s, cuda_status(e));
    const int tiles = s->geo_fused.gx * s->geo_fused.gy;
    size_t liq = 0, tot = (size_t)tiles * s->nz;
    for (size_t q = 0; q < tot && q < nmap; q++) liq += h[q] != 0;
    const double f = tot ? (double)liq / (double)tot : 0.0;
    const size_t n = s->ncell();
    const double need = n < kAutoSmallCells ? 0.0 : (n < kAutoLargeCells ? kAutoLeanFractionMid : kAutoLeanFractionLarge);
    const bool lean = f >= need;
    s->auto_choice = lean ? 0 : 1;
    return PF_OK;
}

template <typename R>
static int do_step(pf_sim *s, int n)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (s->variant == PF_VARIANT_AUTO && s->auto_choice < 0 && cs == cudaStreamCaptureStatusNone) {
        int r = auto_choose<R>(s);
        if (r != PF_OK) return r;
    }
    if (s->prof || !s->use_graphs || cs != cudaStreamCaptureStatusNone || n < 4 || s->direct_steps < 2) {
        int r = do_step_direct<R>(s, n);
        if (r == PF_OK) s->direct_steps += n;
        return r;
    }
    int r = PF_OK;
    if (s->cur != 0) {  // the graph starts from buffer 0
        r = do_step_direct<R>(s, 1);
        if (r != PF_OK) return r;
        n -= 1;
    }
    const int want = use_fused(s) ? 1 : 0;
    if (want) {
        // the graph's fused steps take the liquid maps of both buffers as valid
        cudaError_t e = ensure_maps<R>(s, s->stream);
        if (e != cudaSuccess) return latch(s, cuda_status(e));
    }
    if (want && s->lean_ok) ensure_aux(s);  // before the capture: the graph holds the fork and the join
    if (!s->graph || s->graph_variant != want) {
        if (s->graph) {
            cudaGraphExecDestroy(s->graph);
            s->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return latch(s, cuda_status(e));
        r = do_step_direct<R>(s, 2);  // recorded, not run: buffers end where they started
        e = cudaStreamEndCapture(s->stream, &g);
        if (r != PF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return latch(s, r != PF_OK ? r : cuda_status(e));
        }
        // the kernel nodes' launch priorities (the general planes' sweeps beside the lean kernel) apply
        e = cudaGraphInstantiate(&s->graph, g, s->aux ? cudaGraphInstantiateFlagUseNodePriority : 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            s->graph = nullptr;
            return latch(s, cuda_status(e));
        }
        s->graph_variant = want;
    }
    for (int q = 0; q + 1 < n; q += 2) {
        cudaError_t e = cudaGraphLaunch(s->graph, s->stream);
        if (e != cudaSuccess) return latch(s, cuda_status(e));
    }
    if (n & 1) r = do_step_direct<R>(s, 1);
    return r;
}

template <typename R>
static int do_init(pf_sim *s, uint64_t seed, int ng)
{
    const KParams<R> kp = make_kparams<R>(s);
    const int H = std::min(s->p.seed_layers, s->nz);
    std::vector<double> seeds((size_t)std::max(ng, 1) * 4, 0.0);
    uint64_t stt = seed;
    for (int g = 0; g < ng; g++) {
        seeds[4 * g + 0] = unit53(stt) * (double)s->nx;
        seeds[4 * g + 1] = unit53(stt) * (double)(s->gny > 0 ? s->gny : s->ny);  // a slab: the global domain's rows
        seeds[4 * g + 2] = unit53(stt) * (double)s->p.seed_layers;
        seeds[4 * g + 3] = floor(3.0 * unit53(stt));
    }
    const size_t sb = seeds.size() * sizeof(double);
    if (s->seeds.bytes < sb) {
        dev_free(s->seeds, s->stream);
        int r = dev_alloc(s->seeds, sb, s->stream);
        if (r != PF_OK) return r;
    }
    cudaError_t e = cudaMemcpyAsync(s->seeds.p, seeds.data(), sb, cudaMemcpyHostToDevice, s->stream);
    DevState ds;
    memset(&ds, 0, sizeof ds);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->state.p, &ds, sizeof ds, cudaMemcpyHostToDevice, s->stream);
    s->cur = 0;
    s->tmap_ok[0] = s->tmap_ok[1] = false;
    if (e == cudaSuccess) e = launch_init<R>(kp, s->phi[0].p, s->mu[0].p, (const double *)s->seeds.p, ng, H, s->stream);
    if (e == cudaSuccess && s->comp())
        e = cudaMemsetAsync(s->philo[0].p, 0, s->philo[0].bytes, s->stream);
    if (e == cudaSuccess && s->comp()) e = cudaMemsetAsync(s->mulo[0].p, 0, s->mulo[0].bytes, s->stream);
    if (e == cudaSuccess)
        e = launch_post<R>(kp, (const DevState *)s->state.p, s->phi[0].p, s->mu[0].p, (PlaneT<R> *)s->tab.p,
                           s->stream);
    // the host buffers above are stack/heap locals: wait for the copies before returning
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return latch(s, cuda_status(e));
    s->latched = PF_OK;
    return PF_OK;
}

static const size_t kChunkCells = (size_t)1 << 22;  // staging chunk for host transfers

// host SoA fields of element type H (double or float) <-> the device state, through a staging buffer
// of a chunk of planes
// The device's address of a host buffer it can read and write directly (pinned, mapped host memory:
// on a Grace-Blackwell node the GPU reaches it over NVLink-C2C), else nullptr.
static void *device_view(const void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <typename R, typename H>
static int do_read(pf_sim *s, H *phi, H *mu)
{
    const KParams<R> kp = make_kparams<R>(s);
    const size_t plane = (size_t)s->nx * s->ny, n = s->ncell();
    // host buffers the device can address: one pass of the pack kernel writes them directly
    H *vphi = (H *)device_view(phi), *vmu = (H *)device_view(mu);
    if ((!phi || vphi) && (!mu || vmu)) {
        cudaError_t e = launch_pack<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p, vphi, vmu,
                                       0, s->nz, s->stream, s->lo_phi(s->cur), s->lo_mu(s->cur));
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        return e == cudaSuccess ? PF_OK : latch(s, cuda_status(e));
    }
    int pk = (int)std::max<size_t>(1, std::min<size_t>(s->nz, kChunkCells / plane));
    DevBuf stg;
    int r = dev_alloc(stg, (size_t)pk * plane * 6 * sizeof(H), s->stream);
    if (r != PF_OK) return r;
    H *dphi = (H *)stg.p, *dmu = dphi + (size_t)pk * plane * 4;
    cudaError_t e = cudaSuccess;
    for (int k0 = 0; k0 < s->nz && e == cudaSuccess; k0 += pk) {
        const int nk = std::min(pk, s->nz - k0);
        const size_t m = (size_t)nk * plane;
        e = launch_pack<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p, phi ? dphi : nullptr,
                           mu ? dmu : nullptr, k0, nk, s->stream, s->lo_phi(s->cur), s->lo_mu(s->cur));
        for (int c = 0; c < 4 && phi && e == cudaSuccess; c++)
            e = cudaMemcpyAsync(phi + (size_t)c * n + (size_t)k0 * plane, dphi + (size_t)c * m, m * sizeof(H),
                                cudaMemcpyDeviceToHost, s->stream);
        for (int c = 0; c < 2 && mu && e == cudaSuccess; c++)
            e = cudaMemcpyAsync(mu + (size_t)c * n + (size_t)k0 * plane, dmu + (size_t)c * m, m * sizeof(H),
                                cudaMemcpyDeviceToHost, s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    dev_free(stg, s->stream);
    return e == cudaSuccess ? PF_OK : latch(s, cuda_status(e));
}

template <typename R, typename H>
static int do_write(pf_sim *s, const H *phi, const H *mu)
{
    const KParams<R> kp = make_kparams<R>(s);
    const size_t plane = (size_t)s->nx * s->ny, n = s->ncell();
    // host buffers the device can address: one pass of the unpack kernel reads them directly
    const H *vphi = (const H *)device_view(phi), *vmu = (const H *)device_view(mu);
    if (vphi && vmu) {
        s->tmap_ok[0] = s->tmap_ok[1] = false;
        cudaError_t e = launch_unpack<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p, vphi,
                                         vmu, 0, s->nz, s->stream, s->lo_phi(s->cur), s->lo_mu(s->cur));
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        return e == cudaSuccess ? PF_OK : latch(s, cuda_status(e));
    }
    int pk = (int)std::max<size_t>(1, std::min<size_t>(s->nz, kChunkCells / plane));
    DevBuf stg;
    int r = dev_alloc(stg, (size_t)pk * plane * 6 * sizeof(H), s->stream);
    if (r != PF_OK) return r;
    H *dphi = (H *)stg.p, *dmu = dphi + (size_t)pk * plane * 4;
    cudaError_t e = cudaSuccess;
    s->tmap_ok[0] = s->tmap_ok[1] = false;
    for (int k0 = 0; k0 < s->nz && e == cudaSuccess; k0 += pk) {
        const int nk = std::min(pk, s->nz - k0);
        const size_t m = (size_t)nk * plane;
        for (int c = 0; c < 4 && e == cudaSuccess; c++)
            e = cudaMemcpyAsync(dphi + (size_t)c * m, phi + (size_t)c * n + (size_t)k0 * plane, m * sizeof(H),
                                cudaMemcpyHostToDevice, s->stream);
        for (int c = 0; c < 2 && e == cudaSuccess; c++)
            e = cudaMemcpyAsync(dmu + (size_t)c * m, mu + (size_t)c * n + (size_t)k0 * plane, m * sizeof(H),
                                cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = launch_unpack<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p, dphi, dmu, k0,
                                 nk, s->stream, s->lo_phi(s->cur), s->lo_mu(s->cur));
        // the staging buffer is reused by the next chunk
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    dev_free(stg, s->stream);
    return e == cudaSuccess ? PF_OK : latch(s, cuda_status(e));
}

// The plane table of the current clock and window (no shift pending), after the state was put back.
template <typename R>
static int rebuild_table(pf_sim *s, cudaStream_t st)
{
    const KParams<R> kp = make_kparams<R>(s);
    const cudaError_t e = launch_post<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p,
                                         (PlaneT<R> *)s->tab.p, st, s->lo_phi(s->cur), s->lo_mu(s->cur));
    return e == cudaSuccess ? PF_OK : cuda_status(e);
}

template <typename R>
static int do_reduce(pf_sim *s, double out[8])
{
    const KParams<R> kp = make_kparams<R>(s);
    cudaError_t e = launch_reduce<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p,
                                     (double *)s->red.p, s->stream, s->lo_phi(s->cur), s->lo_mu(s->cur));
    std::vector<double> h((size_t)s->nz * 8);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), s->red.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return latch(s, cuda_status(e));
    for (int q = 0; q < 8; q++) out[q] = 0.0;
    for (int k = 0; k < s->nz; k++)
        for (int q = 0; q < 8; q++) out[q] += h[(size_t)k * 8 + q];
    return PF_OK;
}

// interface mesh of one phase: triangles per segment of cubes, a device scan into the offsets of
// the non-empty segments, the totals to the host, then the triangles of those segments into a
// device buffer copied to the caller's
template <typename R>
static int do_mesh(pf_sim *s, int phase, double iso, float *tris, size_t cap, size_t *ntris)
{
    *ntris = 0;
    if (s->nz < 2) return PF_OK;
    const KParams<R> kp = make_kparams<R>(s);
    const size_t nb = ((size_t)s->nx + 255) / 256, nseg = nb * s->ny * (size_t)(s->nz - 1);
    const size_t npad = (nseg + 15) / 16 * 16;
    // ne_off (npad u64) | totals (2 u64) | counts (npad u32) | ne_seg (npad u32)
    DevBuf scratch;
    int r = dev_alloc(scratch, npad * 8 + 16 + npad * 8, s->stream);
    if (r != PF_OK) return r;
    unsigned long long *ne_off = (unsigned long long *)scratch.p, *dtot = ne_off + npad;
    unsigned *counts = (unsigned *)(dtot + 2), *ne_seg = counts + npad;
    unsigned long long tot[2] = {0, 0};
    cudaError_t e = cudaSuccess;
    if (npad > nseg) e = cudaMemsetAsync(counts + nseg, 0, (npad - nseg) * sizeof(unsigned), s->stream);
    if (e == cudaSuccess)
        e = timed(s, PF_K_MESH_COUNT, [&] {
            return launch_mesh_count<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, phase, iso, counts,
                                        s->stream);
        });
    if (e == cudaSuccess)
        e = timed(s, PF_K_MESH_SCAN, [&] { return launch_mesh_scan<R>(counts, npad, ne_seg, ne_off, dtot, s->stream); });
    if (e == cudaSuccess) e = cudaMemcpyAsync(tot, dtot, sizeof tot, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        dev_free(scratch, s->stream);
        return latch(s, cuda_status(e));
    }
    *ntris = (size_t)tot[0];
    if (!tris || tot[0] == 0) {
        dev_free(scratch, s->stream);
        return PF_OK;
    }
    if (cap < tot[0]) {
        dev_free(scratch, s->stream);
        return PF_E_INVAL;
    }
    DevBuf out;
    r = dev_alloc(out, (size_t)tot[0] * 9 * sizeof(float), s->stream);
    if (r != PF_OK) {
        dev_free(scratch, s->stream);
        return r;
    }
    e = timed(s, PF_K_MESH_EMIT, [&] {
        return launch_mesh_emit<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, phase, iso, ne_seg, ne_off,
                                   (unsigned)tot[1], tot[0], (float *)out.p, s->stream);
    });
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tris, out.p, (size_t)tot[0] * 9 * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    dev_free(out, s->stream);
    dev_free(scratch, s->stream);
    return e == cudaSuccess ? PF_OK : latch(s, cuda_status(e));
}

static int read_state(pf_sim *s, DevState *ds)
{
    cudaError_t e = cudaMemcpyAsync(ds, s->state.p, sizeof *ds, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? PF_OK : latch(s, cuda_status(e));
}

// ------------------------------------------------------------------------------------------
// checkpoints (the paper's infrequent field checkpoints, Section 3.2)
// ------------------------------------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];    // "PFCKPT01"
    int32_t version;  // 1
    int32_t nx, ny, nz;
    int32_t elem;       // bytes per value: 4 (FP32) or 8 (FP64)
    int32_t precision;  // PF_FP64 / PF_FP32 / PF_FP32_COMP of the writer
    int32_t nshift;     // planes shifted since init
    int32_t auto_path;  // PF_VARIANT_AUTO's choice of the writer's run: 0 not made, 1 the lean path
                        // (the default rule), 2 the two whole-domain sweeps
    double t, off;      // simulation time, window offset
    int32_t pad[2];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header");
const char kCkptMagic[8] = {'P', 'F', 'C', 'K', 'P', 'T', '0', '1'};
}  // namespace

template <typename R>
static int do_checkpoint_write(pf_sim *s, const char *path, int single)
{
    DevState ds;
    int r = read_state(s, &ds);
    if (r != PF_OK) return r;
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.nx = s->nx;
    h.ny = s->ny;
    h.nz = s->nz;
    // the state's own values, exactly: FP32 words for FP32, FP64 for FP64, and for the compensated
    // state its two FP32 words (a high/low pair need not be one FP64 value)
    // (single: the paper's single-precision checkpoint, every value rounded once to FP32 and written as
    // an FP32 writer's file)
    const bool pairs = s->comp() && !single;
    h.elem = s->p.precision == PF_FP64 && !single ? 8 : 4;
    h.precision = single ? PF_FP32 : s->p.precision;
    h.nshift = ds.nshift_total;
    h.auto_path = s->auto_choice + 1;
    h.t = ds.t;
    h.off = ds.off;
    const KParams<R> kp = make_kparams<R>(s);
    const size_t plane = (size_t)s->nx * s->ny;
    const int pk = (int)std::max<size_t>(1, std::min<size_t>(s->nz, kChunkCells / plane));
    DevBuf stg;
    r = dev_alloc(stg, (size_t)pk * plane * 6 * sizeof(double), s->stream);
    if (r != PF_OK) return r;
    FILE *f = fopen(path, "wb");
    if (!f) {
        dev_free(stg, s->stream);
        return PF_E_INVAL;
    }
    bool io_ok = fwrite(&h, sizeof h, 1, f) == 1;
    const int nwords = pairs ? 2 : 1;  // word 0: the values (high words); word 1: the low words
    std::vector<double> hb((size_t)nwords * pk * plane * 6);
    std::vector<float> hf(h.elem == 4 ? plane : 0);
    double *dphi = (double *)stg.p, *dmu = dphi + (size_t)pk * plane * 4;
    cudaError_t e = cudaSuccess;
    for (int k0 = 0; k0 < s->nz && e == cudaSuccess && io_ok; k0 += pk) {
        const int nk = std::min(pk, s->nz - k0);
        const size_t m = (size_t)nk * plane;
        for (int w = 0; w < nwords && e == cudaSuccess; w++) {
            // each word array alone (the low words packed as if they were the fields): exact in FP64
            double *hw = hb.data() + (size_t)w * m * 6;
            e = launch_pack<R>(kp, (const DevState *)s->state.p, w ? s->philo[s->cur].p : s->phi[s->cur].p,
                               w ? s->mulo[s->cur].p : s->mu[s->cur].p, dphi, dmu, k0, nk, s->stream,
                               pairs ? nullptr : s->lo_phi(s->cur), pairs ? nullptr : s->lo_mu(s->cur));
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hw, dphi, m * 4 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hw + m * 4, dmu, m * 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        }
        for (int kk = 0; kk < nk && e == cudaSuccess && io_ok; kk++)
            for (int w = 0; w < nwords && io_ok; w++)
                for (int c = 0; c < 6 && io_ok; c++) {
                    const double *src = hb.data() + (size_t)w * m * 6 + (size_t)c * m + (size_t)kk * plane;
                    if (h.elem == 4) {
                        for (size_t q = 0; q < plane; q++) hf[q] = (float)src[q];
                        io_ok = fwrite(hf.data(), sizeof(float), plane, f) == plane;
                    } else {
                        io_ok = fwrite(src, sizeof(double), plane, f) == plane;
                    }
                }
    }
    io_ok = (fclose(f) == 0) && io_ok;
    dev_free(stg, s->stream);
    if (e != cudaSuccess) return latch(s, cuda_status(e));
    return io_ok ? PF_OK : PF_E_INVAL;
}

template <typename R>
static int do_checkpoint_read(pf_sim *s, const char *path)
{
    FILE *f = fopen(path, "rb");
    if (!f) return PF_E_INVAL;
    CkptHeader h;
    bool io_ok = fread(&h, sizeof h, 1, f) == 1;
    if (!io_ok || memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1 || h.nx != s->nx || h.ny != s->ny ||
        h.nz != s->nz || (h.elem != 4 && h.elem != 8)) {
        fclose(f);
        return PF_E_INVAL;
    }
    const KParams<R> kp = make_kparams<R>(s);
    const size_t plane = (size_t)s->nx * s->ny;
    const int pk = (int)std::max<size_t>(1, std::min<size_t>(s->nz, kChunkCells / plane));
    DevBuf stg;
    int r = dev_alloc(stg, (size_t)pk * plane * 6 * sizeof(double), s->stream);
    if (r != PF_OK) {
        fclose(f);
        return r;
    }
    // a compensated writer stored both FP32 words of each value (high arrays, then low arrays, per plane)
    const bool file_pairs = h.precision == PF_FP32_COMP && h.elem == 4;
    const int nwords = file_pairs ? 2 : 1;
    std::vector<double> hb((size_t)nwords * pk * plane * 6);
    std::vector<float> hf(h.elem == 4 ? plane : 0);
    double *dphi = (double *)stg.p, *dmu = dphi + (size_t)pk * plane * 4;
    cudaError_t e = cudaSuccess;
    s->tmap_ok[0] = s->tmap_ok[1] = false;
    for (int k0 = 0; k0 < s->nz && e == cudaSuccess && io_ok; k0 += pk) {
        const int nk = std::min(pk, s->nz - k0);
        const size_t m = (size_t)nk * plane;
        for (int kk = 0; kk < nk && io_ok; kk++)
            for (int w = 0; w < nwords && io_ok; w++)
                for (int c = 0; c < 6 && io_ok; c++) {
                    double *dst = hb.data() + (size_t)w * m * 6 + (size_t)c * m + (size_t)kk * plane;
                    if (h.elem == 4) {
                        io_ok = fread(hf.data(), sizeof(float), plane, f) == plane;
                        for (size_t q = 0; q < plane && io_ok; q++) dst[q] = (double)hf[q];
                    } else {
                        io_ok = fread(dst, sizeof(double), plane, f) == plane;
                    }
                }
        if (!io_ok) break;
        if (file_pairs && !s->comp())  // into another precision: the value of each pair, rounded once
            for (size_t q = 0; q < m * 6; q++) hb[q] += hb[m * 6 + q];
        // a compensated reader of pairs takes both words as they are; otherwise the values
        const int nw = file_pairs && s->comp() ? 2 : 1;
        for (int w = 0; w < nw && e == cudaSuccess; w++) {
            const double *hw = hb.data() + (size_t)w * m * 6;
            e = cudaMemcpyAsync(dphi, hw, m * 4 * sizeof(double), cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dmu, hw + m * 4, m * 2 * sizeof(double), cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) {
                if (nw == 2)
                    e = launch_unpack<R>(kp, (const DevState *)s->state.p, w ? s->philo[s->cur].p : s->phi[s->cur].p,
                                         w ? s->mulo[s->cur].p : s->mu[s->cur].p, dphi, dmu, k0, nk, s->stream,
                                         nullptr, nullptr);
                else
                    e = launch_unpack<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p, dphi,
                                         dmu, k0, nk, s->stream, s->lo_phi(s->cur), s->lo_mu(s->cur));
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // the host chunk is reused
        }
    }
    fclose(f);
    if (e == cudaSuccess && io_ok) {
        // the clock and window of the checkpoint; no shift pending; the plane table for them
        DevState ds;
        r = read_state(s, &ds);
        if (r != PF_OK) {
            dev_free(stg, s->stream);
            return r;
        }
        ds.t = h.t;
        ds.off = h.off;
        ds.shift = 0;
        ds.nonfinite = 0;
        ds.nshift_total = h.nshift;
        // the writer's run's choice of path continues (a file without one: chosen at the next step)
        s->auto_choice = h.auto_path == 1 || h.auto_path == 2 ? h.auto_path - 1 : -1;
        e = cudaMemcpyAsync(s->state.p, &ds, sizeof ds, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = launch_post<R>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p,
                               (PlaneT<R> *)s->tab.p, s->stream, s->lo_phi(s->cur), s->lo_mu(s->cur));
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    }
    dev_free(stg, s->stream);
    if (e != cudaSuccess) return latch(s, cuda_status(e));
    return io_ok ? PF_OK : PF_E_INVAL;
}

#define PF_DISPATCH(s, fn, ...) ((s)->p.precision == PF_FP64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
extern "C" {

const char *pf_strerror(int st)
{
    switch (st) {
    case PF_OK: return "ok";
    case PF_E_INVAL: return "invalid argument";
    case PF_E_NOMEM: return "out of memory (or admission refused)";
    case PF_E_CUDA: return "CUDA error";
    case PF_E_UNSTABLE: return "non-finite value in phi or mu";
    case PF_E_TIMEOUT: return "timed out";
    case PF_E_CANCELLED: return "cancelled";
    case PF_E_PENDING: return "pending";
    default: return "unknown status";
    }
}

int pf_default_params(pf_params *p)
{
    if (!p) return PF_E_INVAL;
    memset(p, 0, sizeof *p);
    p->version = PF_PARAMS_VERSION;
    p->precision = PF_FP64;
    p->dx = 1.0;
    p->eps = 4.0;
    p->tau = 1.0;
    p->dt = 0.0;
    for (int q = 0; q < 6; q++) p->gamma2[q] = 1.0;
    for (int q = 0; q < 4; q++) p->gamma3[q] = 15.0;
    const double cE[4][2] = {{0.8, 0.1}, {0.1, 0.8}, {0.1, 0.1}, {1.0 / 3.0, 1.0 / 3.0}};
    for (int a = 0; a < 4; a++) {
        p->A[a] = 1.0;
        p->cE[a][0] = cE[a][0];
        p->cE[a][1] = cE[a][1];
        p->kT[a][0] = p->kT[a][1] = a == 3 ? 0.1 : 0.0;
        p->s[a] = a == 3 ? 0.0 : 1.0;
        p->D[a] = a == 3 ? 1.0 : 0.0;
    }
    p->TE = 1.0;
    p->G = 1e-3;
    p->v = 1e-2;
    p->seed_layers = 8;
    p->T0 = p->TE - p->G * (double)p->seed_layers - 0.15;  // the seeds start 0.15 below TE
    p->n_grains = 12;
    p->window_trigger_z = 0.0;
    return PF_OK;
}

int pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return PF_E_INVAL;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return PF_OK;
}

int pf_destroy(pf_sim *s)
{
    if (!s) return PF_E_INVAL;
    cudaStreamSynchronize(s->stream);
    for (int b = 0; b < 2; b++) {
        dev_free(s->phi[b], s->stream);
        dev_free(s->mu[b], s->stream);
        dev_free(s->philo[b], s->stream);
        dev_free(s->mulo[b], s->stream);
        dev_free(s->tmap[b], s->stream);
    }
    dev_free(s->state, s->stream);
    dev_free(s->parts, s->stream);
    dev_free(s->lean_stats, s->stream);
    dev_free(s->splits, s->stream);
    dev_free(s->glist, s->stream);
    dev_free(s->subparts, s->stream);
    dev_free(s->subcnt, s->stream);
    dev_free(s->tab, s->stream);
    dev_free(s->seeds, s->stream);
    dev_free(s->red, s->stream);
    for (auto &r : s->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : s->pool) cudaEventDestroy(e);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    if (s->aux) {
        cudaStreamSynchronize(s->aux);
        cudaStreamDestroy(s->aux);
    }
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return PF_OK;
}

int pf_create(int nx, int ny, int nz, const pf_params *p, void *stream, pf_sim **out)
{
    if (!out) return PF_E_INVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return PF_E_INVAL;
    if ((size_t)nx * ny > (size_t)1 << 31 || (size_t)nz > (size_t)1 << 24) return PF_E_INVAL;
    int r = check_params(p);
    if (r != PF_OK) return r;
    pf_sim *s = new (std::nothrow) pf_sim;
    if (!s) return PF_E_NOMEM;
    s->nx = nx;
    s->ny = ny;
    s->nz = nz;
    s->p = *p;
    if (!(s->p.dt > 0.0)) s->p.dt = default_dt(s->p, nz);
    if (stream) {
        s->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete s;
            return cuda_status(e);
        }
        s->own_stream = true;
    }
    s->geo = make_geometry(nx, ny, nz, 0);
    {
        // fused: about 6 CTAs per SM in total, 32..256 planes per CTA
        const long tiles = (long)s->geo.gx * s->geo.gy;
        long chunks = (152L * 6 + tiles - 1) / tiles;
        int zc = (int)((nz + chunks - 1) / chunks);
        zc = std::max(32, std::min(256, zc));
        s->geo_fused = make_geometry(nx, ny, nz, zc);
    }
    const size_t n = s->ncell(), w = s->wbytes();
    const size_t tabsz = (size_t)2 * nz * 16 * w;
    for (int b = 0; b < 2 && r == PF_OK; b++) {
        r = dev_alloc(s->phi[b], n * 4 * w, s->stream);
        if (r == PF_OK) r = dev_alloc(s->mu[b], n * 2 * w, s->stream);
        if (r == PF_OK && s->comp()) r = dev_alloc(s->philo[b], n * 4 * w, s->stream);
        if (r == PF_OK && s->comp()) r = dev_alloc(s->mulo[b], n * 2 * w, s->stream);
    }
    for (int b = 0; b < 2 && r == PF_OK; b++)
        r = dev_alloc(s->tmap[b], (size_t)nz * s->geo_fused.gx * s->geo_fused.gy, s->stream);
    if (r == PF_OK) r = dev_alloc(s->state, sizeof(DevState), s->stream);
    // lean CTAs: at most PF_LEAN_PLANES planes each
    s->lean_nsub = std::max(1, (s->geo_fused.zchunk + PF_LEAN_PLANES - 1) / PF_LEAN_PLANES);
    if (r == PF_OK)
        r = dev_alloc(s->parts, (size_t)std::max(s->geo.nparts(), s->geo_fused.nparts()) * sizeof(Partial),
                      s->stream);
    if (r == PF_OK) r = dev_alloc(s->lean_stats, sizeof(LeanStats), s->stream);
    if (r == PF_OK) r = dev_alloc(s->splits, (size_t)s->geo_fused.nparts() * sizeof(int2), s->stream);
    {
        // work units of the general planes: up to kMaxUnits per item
        const size_t units = (size_t)s->geo_fused.nparts() * kMaxUnits;
        if (r == PF_OK) r = dev_alloc(s->glist, (size_t)s->geo_fused.nparts() * sizeof(int), s->stream);
        if (r == PF_OK) r = dev_alloc(s->subparts, units * sizeof(Partial), s->stream);
        if (r == PF_OK) r = dev_alloc(s->subcnt, (size_t)s->geo_fused.nparts() * sizeof(unsigned), s->stream);
        if (r == PF_OK) {
            cudaError_t e = cudaMemsetAsync(s->subcnt.p, 0, s->subcnt.bytes, s->stream);
            if (e != cudaSuccess) r = cuda_status(e);
        }
    }
    if (r == PF_OK) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // persistent general CTAs: PF_GENERAL_CTAS_PER_SM per SM, at most what fits (two take all of
        // an SM's registers; the lean CTAs beside them get SMs as general CTAs finish)
        const int per_sm = std::min(PF_GENERAL_CTAS_PER_SM, p->precision == PF_FP64 ? general_ctas_per_sm<double>()
                                                                                    : general_ctas_per_sm<float>());
        s->general_ctas = std::max(1, std::min(s->geo_fused.nparts(), per_sm * sms));
        int pp = 1, pm = 1;
        if (p->precision == PF_FP64)
            general_sweep_ctas_per_sm<double>(&pp, &pm);
        else
            general_sweep_ctas_per_sm<float>(&pp, &pm);
        const int units = s->geo_fused.nparts() * kMaxUnits;
        s->gphi_ctas = std::max(1, std::min(units, std::min(pp, PF_GENERAL_CTAS_PER_SM) * sms));
        s->gmu_ctas = std::max(1, std::min(units, std::min(pm, PF_GENERAL_CTAS_PER_SM) * sms));
    }
    if (r == PF_OK) {
        cudaError_t e = cudaMemsetAsync(s->lean_stats.p, 0, sizeof(LeanStats), s->stream);
        if (e != cudaSuccess) r = cuda_status(e);
    }
    if (r == PF_OK) {
        // the lean kernel's tensor maps of the two mu buffers (the compensated state: its high words)
        s->lean_ok = true;
        for (int b = 0; b < 2; b++)
            s->lean_ok = s->lean_ok && encode_lean_maps(&s->mu_map[b], s->mu[b].p, nx, ny, nz, w, s->geo_fused.tx,
                                                     s->geo_fused.ty);
    }
    if (r == PF_OK) r = dev_alloc(s->tab, tabsz, s->stream);
    if (r == PF_OK) r = dev_alloc(s->red, (size_t)nz * 8 * sizeof(double), s->stream);
    if (r != PF_OK) {
        pf_destroy(s);
        return r;
    }
    // pure liquid, mu = 0, t = 0 until pf_init / pf_write_fields
    r = PF_DISPATCH(s, do_init, s, (uint64_t)0, 0);
    if (r != PF_OK) {
        pf_destroy(s);
        return r;
    }
    *out = s;
    return PF_OK;
}

int pf_get_params(const pf_sim *s, pf_params *out)
{
    if (!s || !out) return PF_E_INVAL;
    *out = s->p;
    return PF_OK;
}

int pf_init(pf_sim *s, uint64_t seed)
{
    if (!s) return PF_E_INVAL;
    s->auto_choice = -1;
    return PF_DISPATCH(s, do_init, s, seed, s->p.n_grains);
}

int pf_step(pf_sim *s, int nsteps)
{
    if (!s || nsteps < 0) return PF_E_INVAL;
    if (s->latched != PF_OK) return s->latched;
    if (nsteps == 0) return PF_OK;
    return PF_DISPATCH(s, do_step, s, nsteps);
}

int pf_sync(pf_sim *s)
{
    if (!s) return PF_E_INVAL;
    DevState ds;
    int r = read_state(s, &ds);
    if (r == PF_OK && ds.nonfinite) latch(s, ds.nonfinite == 2 ? PF_E_TIMEOUT : PF_E_UNSTABLE);
    r = s->latched;
    s->latched = PF_OK;
    if (r == PF_E_UNSTABLE || r == PF_E_TIMEOUT) {
        // clear the sticky device flag with the latched error
        ds.nonfinite = 0;
        cudaMemcpyAsync(s->state.p, &ds, sizeof ds, cudaMemcpyHostToDevice, s->stream);
        cudaStreamSynchronize(s->stream);
    }
    return r;
}

int pf_read_fields(pf_sim *s, double *phi, double *mu, size_t cap_cells)
{
    if (!s || cap_cells < s->ncell()) return PF_E_INVAL;
    if (!phi && !mu) return PF_OK;
    return PF_DISPATCH(s, do_read, s, phi, mu);
}

int pf_write_fields(pf_sim *s, const double *phi, const double *mu)
{
    if (!s || !phi || !mu) return PF_E_INVAL;
    s->auto_choice = -1;
    return PF_DISPATCH(s, do_write, s, phi, mu);
}

int pf_read_fields_f32(pf_sim *s, float *phi, float *mu, size_t cap_cells)
{
    if (!s || cap_cells < s->ncell()) return PF_E_INVAL;
    if (!phi && !mu) return PF_OK;
    return PF_DISPATCH(s, do_read, s, phi, mu);
}

int pf_write_fields_f32(pf_sim *s, const float *phi, const float *mu)
{
    if (!s || !phi || !mu) return PF_E_INVAL;
    s->auto_choice = -1;
    return PF_DISPATCH(s, do_write, s, phi, mu);
}

int pf_checkpoint_write(pf_sim *s, const char *path)
{
    if (!s || !path) return PF_E_INVAL;
    return PF_DISPATCH(s, do_checkpoint_write, s, path, 0);
}

int pf_checkpoint_write_f32(pf_sim *s, const char *path)
{
    if (!s || !path) return PF_E_INVAL;
    return PF_DISPATCH(s, do_checkpoint_write, s, path, 1);
}

int pf_checkpoint_read(pf_sim *s, const char *path)
{
    if (!s || !path) return PF_E_INVAL;
    return PF_DISPATCH(s, do_checkpoint_read, s, path);
}

int pf_interface_mesh(pf_sim *s, int phase, double iso, float *tris, size_t cap_tris, size_t *ntris)
{
    if (!s || !ntris || phase < 0 || phase > 3 || !isfinite(iso)) return PF_E_INVAL;
    return PF_DISPATCH(s, do_mesh, s, phase, iso, tris, cap_tris, ntris);
}

int pf_phase_fractions(pf_sim *s, double out[4])
{
    if (!s || !out) return PF_E_INVAL;
    double acc[8];
    int r = PF_DISPATCH(s, do_reduce, s, acc);
    if (r != PF_OK) return r;
    for (int a = 0; a < 4; a++) out[a] = acc[a] / (double)s->ncell();
    return PF_OK;
}

int pf_stats(pf_sim *s, double *t, double *off, double solute[2], double *h_int)
{
    if (!s) return PF_E_INVAL;
    double acc[8];
    int r = PF_DISPATCH(s, do_reduce, s, acc);
    if (r != PF_OK) return r;
    DevState ds;
    r = read_state(s, &ds);
    if (r != PF_OK) return r;
    if (t) *t = ds.t;
    if (off) *off = ds.off;
    if (solute) {
        solute[0] = acc[4];
        solute[1] = acc[5];
    }
    if (h_int) *h_int = acc[6] / ((double)s->nx * (double)s->ny);
    return PF_OK;
}

int pf_window_shifts(pf_sim *s, int *planes)
{
    if (!s || !planes) return PF_E_INVAL;
    DevState ds;
    int r = read_state(s, &ds);
    if (r != PF_OK) return r;
    *planes = ds.nshift_total;
    return PF_OK;
}

int pf_step_bytes(pf_sim *s, double bytes[])
{
    if (!s || !bytes) return PF_E_INVAL;
    for (int c = 0; c < PF_K_COUNT; c++) bytes[c] = 0.0;
    if (s->last_kind < 0) return PF_OK;
    const double cells = (double)s->ncell(), w = (double)s->wbytes();
    if (s->last_kind == 0) {
        // phi-sweep: phi^n, mu^n in, phi^{n+1} out (10 words; 18 with the compensated low words of
        // phi in and out); mu-sweep: phi^n, phi^{n+1}, mu^n in, mu^{n+1} out (12 words; 16)
        bytes[PF_K_PHI] = cells * w * (s->comp() ? 18.0 : 10.0);
        bytes[PF_K_MU] = cells * w * (s->comp() ? 16.0 : 12.0);
        return PF_OK;
    }
    std::vector<Partial> h((size_t)s->last_nparts);
    LeanStats ls;
    memset(&ls, 0, sizeof ls);
    cudaError_t e = cudaMemcpyAsync(h.data(), s->parts.p, h.size() * sizeof(Partial), cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess && s->last_kind == 2)
        e = cudaMemcpyAsync(&ls, s->lean_stats.p, sizeof ls, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return latch(s, cuda_status(e));
    double g = 0.0;
    for (const Partial &x : h) g += x.bytes;
    bytes[s->last_kind == 2 && PF_GENERAL_SWEEPS ? PF_K_GENERAL : PF_K_FUSED] = g;
    bytes[PF_K_LEAN] = (double)ls.last_bytes;
    return PF_OK;
}

int pf_test_withhold_copies(pf_sim *s, int on)
{
    if (!s) return PF_E_INVAL;
    s->test_withhold = on != 0;
    if (s->graph) {  // captured with the previous parameters
        cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
    }
    return PF_OK;
}

int pf_set_variant(pf_sim *s, int variant)
{
    if (!s || variant < PF_VARIANT_AUTO || variant > PF_VARIANT_FUSED) return PF_E_INVAL;
    s->variant = variant;
    s->auto_choice = -1;  // AUTO chooses again from the state at the next step
    return PF_OK;
}

int pf_profile(pf_sim *s, int enable)
{
    if (!s) return PF_E_INVAL;
    s->prof = enable != 0;
    return PF_OK;
}

int pf_profile_read(pf_sim *s, double ms[], int launches[])
{
    if (!s || !ms || !launches) return PF_E_INVAL;
    for (int c = 0; c < PF_K_COUNT; c++) {
        ms[c] = 0.0;
        launches[c] = 0;
    }
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return latch(s, cuda_status(e));
    for (auto &r : s->recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.cls >= 0 && r.cls < PF_K_COUNT) {
            ms[r.cls] += (double)t;
            launches[r.cls] += 1;
        }
        s->pool.push_back(r.a);
        s->pool.push_back(r.b);
    }
    s->recs.clear();
    return PF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// batched launch
// ------------------------------------------------------------------------------------------
struct pf_batch {
    std::vector<pf_sim *> sims;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int precision = PF_FP32;
    int zchunk = 0;
    int general_per_sm = PF_GENERAL_CTAS_PER_SM;  // persistent general CTAs per SM (autotuned)
    int lean_split = 1;  // lean CTAs per z chunk: this many times the fewest that keep <= 64 planes a CTA (autotuned)
    int lean_rows = 8;   // rows of a lean CTA's tile: 8 (a liquid-map tile) or 4 (half of one) (autotuned)
    DevBuf doms;     // BatchDomain<R>[n]
    DevBuf items;    // BatchItem[nitems]
    DevBuf parts;    // Partial[sum of tiles]
    DevBuf counter;  // work-item counter
    int nitems = 0, ctas = 0, post_blocks = 1;
    bool built = false;
    cudaGraphExec_t graph = nullptr;
    int direct_steps = 0;
    // descriptors are built relative to each domain's current buffer: parity counts the steps since
    // the build (mod 2); cur0 holds each domain's buffer index at the build
    int parity = 0;
    std::vector<int> cur0;
    size_t dom_capacity = 0;
    bool owns_sims = true;
    // lean path (domains with TMA maps): plan entries (domain, item), lean items (domain, tile x,
    // tile y, chunk * nsub + sub), the splits of all its domains, the batch-wide general list and its
    // counters; the other domains run the fused tile over `items`
    DevBuf plan_entries, lean_items, splits, glist, plan;
    int nplan = 0, nlean = 0, gphi_ctas = 1, gmu_ctas = 1;
    bool lean_mode = false;
    bool sym = true;  // every domain has the symmetric set (no matrix curvature, no pair times)
    size_t nparts_total = 0;  // partial sums of all domains (their algorithmic-byte tallies)
    // the general planes' sweeps beside the lean kernel (as a single domain's, PF_CONCURRENT)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<char> dom_lean;  // the domain runs the lean path
};

template <typename R>
static int batch_build(pf_batch *b)
{
    const int n = (int)b->sims.size();
    std::vector<BatchDomain<R>> d(n);
    std::vector<size_t> part_off(n), split_off(n);
    std::vector<BatchItem> items;
    std::vector<std::pair<long, int>> order;  // (cost, item) for the largest-first sort
    std::vector<int2> plan_entries;
    std::vector<int4> lean_items;
    std::vector<std::pair<long, int>> lean_order;  // (domain cells, domain) for the lean items' order
    size_t part_total = 0, split_total = 0;
    int post = 1;
    for (int q = 0; q < n; q++) {
        pf_sim *s = b->sims[q];
        int zc = b->zchunk;
        if (zc <= 0) zc = s->geo_fused.zchunk;
        const Geometry g = make_geometry(s->nx, s->ny, s->nz, zc);
        KParams<R> kp = make_kparams<R>(s);
        kp.zchunk = g.zchunk;
        d[q].kp = kp;
        if (q == 0) b->sym = true;
        b->sym = b->sym && !kp.gen && !kp.gen_tau;
        for (int k = 0; k < 2; k++) {
            d[q].phi[k] = s->phi[k ^ s->cur].p;
            d[q].mu[k] = s->mu[k ^ s->cur].p;
            d[q].tmap[k] = (unsigned char *)s->tmap[k ^ s->cur].p;
            d[q].mu_map[k] = s->mu_map[k ^ s->cur];
        }
        // half-height lean tiles copy boxes of their own height
        bool maps_ok = true;
        if (b->lean_rows != g.ty)
            for (int k = 0; k < 2; k++)
                maps_ok = maps_ok && encode_lean_maps(&d[q].mu_map[k], s->mu[k ^ s->cur].p, s->nx, s->ny, s->nz,
                                                      sizeof(R), g.tx, b->lean_rows);
        d[q].st = (DevState *)s->state.p;
        d[q].tab = (PlaneT<R> *)s->tab.p;
        d[q].parts = nullptr;  // set once the partial-sum array exists
        d[q].splits = nullptr;
        d[q].lean = nullptr;
        part_off[q] = part_total;
        d[q].gx = g.gx;
        d[q].gy = g.gy;
        d[q].gz = g.gz;
        d[q].nsub = std::min(g.zchunk, std::max(1, (g.zchunk + PF_LEAN_PLANES - 1) / PF_LEAN_PLANES) * b->lean_split);
        part_total += (size_t)g.nparts();
        // the lean path needs the TMA maps and a chunk the batched plan covers
        const bool lean = s->lean_ok && maps_ok && g.zchunk + 4 <= 64 * 9;
        if (q == 0) b->dom_lean.assign(n, 0);
        b->dom_lean[q] = lean ? 1 : 0;
        if (lean) {
            split_off[q] = split_total;
            split_total += (size_t)g.nparts();
            d[q].lean = (LeanStats *)s->lean_stats.p;
            for (int it = 0; it < g.nparts(); it++) plan_entries.push_back(make_int2(q, it));
            lean_order.push_back({(long)s->nx * s->ny * s->nz, q});
        } else {
            for (int bz = 0; bz < g.gz; bz++)
                for (int by = 0; by < g.gy; by++)
                    for (int bx = 0; bx < g.gx; bx++) {
                        const int planes = std::min(g.zchunk, s->nz - bz * g.zchunk);
                        // cost ~ planes + the chunk's two recomputed planes; the chunk at the bottom of
                        // the window holds the solidification front
                        const long cost = (long)(planes + 3) * (bz == 0 ? 4 : 1);
                        order.push_back({cost, (int)items.size()});
                        items.push_back({q, bx, by, bz});
                    }
        }
        const long pw = std::max<long>((long)s->nx * s->ny, 2L * s->nz);
        post = std::max(post, (int)std::min<long>(64, (pw + 255) / 256));
    }
    // lean items of the largest domains first
    std::stable_sort(lean_order.begin(), lean_order.end(),
                     [](const std::pair<long, int> &x, const std::pair<long, int> &y) { return x.first > y.first; });
    for (const auto &lo : lean_order) {
        const int q = lo.second;
        // row blocks of lean_rows rows (those of a map tile share its split)
        const int nby = (b->sims[q]->ny + b->lean_rows - 1) / b->lean_rows;
        for (int z = 0; z < d[q].gz * d[q].nsub; z++)
            for (int by = 0; by < nby; by++)
                for (int bx = 0; bx < d[q].gx; bx++) lean_items.push_back(make_int4(q, bx, by, z));
    }
    std::stable_sort(order.begin(), order.end(), [](const std::pair<long, int> &x, const std::pair<long, int> &y) {
        return x.first > y.first;
    });
    std::vector<BatchItem> sorted(items.size());
    for (size_t q = 0; q < order.size(); q++) sorted[q] = items[order[q].second];
    dev_free(b->items, b->stream);
    dev_free(b->parts, b->stream);
    dev_free(b->plan_entries, b->stream);
    dev_free(b->lean_items, b->stream);
    dev_free(b->splits, b->stream);
    dev_free(b->glist, b->stream);
    int r = dev_alloc(b->items, std::max<size_t>(1, sorted.size()) * sizeof(BatchItem), b->stream);
    if (r == PF_OK) r = dev_alloc(b->parts, std::max<size_t>(1, part_total) * sizeof(Partial), b->stream);
    if (r == PF_OK) r = dev_alloc(b->plan_entries, std::max<size_t>(1, plan_entries.size()) * sizeof(int2), b->stream);
    if (r == PF_OK) r = dev_alloc(b->lean_items, std::max<size_t>(1, lean_items.size()) * sizeof(int4), b->stream);
    if (r == PF_OK) r = dev_alloc(b->splits, std::max<size_t>(1, split_total) * sizeof(int2), b->stream);
    if (r == PF_OK) r = dev_alloc(b->glist, std::max<size_t>(1, plan_entries.size()) * sizeof(int2), b->stream);
    if (r == PF_OK && !b->plan.p) r = dev_alloc(b->plan, sizeof(BatchPlan), b->stream);
    if (r == PF_OK && b->dom_capacity < (size_t)n) {
        dev_free(b->doms, b->stream);
        r = dev_alloc(b->doms, (size_t)n * sizeof(BatchDomain<R>), b->stream);
        b->dom_capacity = r == PF_OK ? (size_t)n : 0;
    }
    if (r == PF_OK && !b->counter.p) r = dev_alloc(b->counter, 256, b->stream);
    if (r != PF_OK) return r;
    for (int q = 0; q < n; q++) {
        d[q].parts = (Partial *)b->parts.p + part_off[q];
        if (d[q].lean) d[q].splits = (int2 *)b->splits.p + split_off[q];
    }
    cudaError_t e = cudaSuccess;
    if (!sorted.empty())
        e = cudaMemcpyAsync(b->items.p, sorted.data(), sorted.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !plan_entries.empty())
        e = cudaMemcpyAsync(b->plan_entries.p, plan_entries.data(), plan_entries.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !lean_items.empty())
        e = cudaMemcpyAsync(b->lean_items.p, lean_items.data(), lean_items.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->doms.p, d.data(), (size_t)n * sizeof(BatchDomain<R>), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // host vectors go out of scope
    if (e != cudaSuccess) return cuda_status(e);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->ctas = std::max(1, std::min((int)std::max<size_t>(1, sorted.size()), fused_ctas_per_sm<R>() * sms));
    b->nitems = (int)sorted.size();
    b->nplan = (int)plan_entries.size();
    b->nlean = (int)lean_items.size();
    b->lean_mode = b->nplan > 0;
    if (b->lean_mode) {
        int pp = 1, pm = 1;
        batched_general_ctas_per_sm<R>(&pp, &pm);
        b->gphi_ctas = std::max(1, std::min(b->nplan, std::min(pp, b->general_per_sm) * sms));
        b->gmu_ctas = std::max(1, std::min(b->nplan, std::min(pm, b->general_per_sm) * sms));
    }
    b->post_blocks = post;
    b->nparts_total = part_total;
    if (PF_CONCURRENT && b->lean_mode && !b->aux) {
        // the second stream and its fork / join events (not while the batch's stream is being
        // captured: such a step runs the general sweeps in line)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            int lo = 0, hi = 0;
            cudaStream_t x = nullptr;
            cudaEvent_t f0 = nullptr, f1 = nullptr;
            cudaError_t ea = cudaDeviceGetStreamPriorityRange(&lo, &hi);
            if (ea == cudaSuccess) ea = cudaStreamCreateWithPriority(&x, cudaStreamNonBlocking, hi);
            if (ea == cudaSuccess) ea = cudaEventCreateWithFlags(&f0, cudaEventDisableTiming);
            if (ea == cudaSuccess) ea = cudaEventCreateWithFlags(&f1, cudaEventDisableTiming);
            if (ea == cudaSuccess) {
                b->aux = x;
                b->ev_fork = f0;
                b->ev_join = f1;
            } else {
                if (x) cudaStreamDestroy(x);
                if (f0) cudaEventDestroy(f0);
                if (f1) cudaEventDestroy(f1);
            }
        }
        cudaGetLastError();
    }
    b->built = true;
    b->parity = 0;
    b->cur0.resize(n);
    for (int q = 0; q < n; q++) b->cur0[q] = b->sims[q]->cur;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return PF_OK;
}

template <typename R>
static int batch_step_direct(pf_batch *b, int n)
{
    for (int q = 0; q < n; q++) {
        cudaError_t e;
        if (b->lean_mode)
            e = launch_batched_lean_step<R>((const BatchDomain<R> *)b->doms.p, (int)b->sims.size(),
                                            (const int2 *)b->plan_entries.p, b->nplan, (const int4 *)b->lean_items.p,
                                            b->nlean, (int2 *)b->glist.p, (BatchPlan *)b->plan.p, b->gphi_ctas,
                                            b->gmu_ctas, (const BatchItem *)b->items.p, b->nitems,
                                            (unsigned *)b->counter.p, b->ctas, b->parity, b->post_blocks, b->stream,
                                            b->sym, b->aux, b->ev_fork, b->ev_join, b->lean_rows);
        else
            e = launch_batched_step<R>((const BatchDomain<R> *)b->doms.p, (int)b->sims.size(),
                                       (const BatchItem *)b->items.p, b->nitems, (unsigned *)b->counter.p, b->parity,
                                       b->ctas, b->post_blocks, b->stream);
        if (e != cudaSuccess) return cuda_status(e);
        b->parity ^= 1;
        for (pf_sim *s : b->sims) {
            s->cur = 1 - s->cur;
            s->tmap_ok[s->cur] = true;  // written by the step's kernels and the window fill
        }
    }
    return PF_OK;
}

template <typename R>
static int batch_step(pf_batch *b, int n)
{
    if (!b->built) {
        int r = batch_build<R>(b);
        if (r != PF_OK) return r;
    }
    for (size_t q = 0; q < b->sims.size(); q++)
        if (b->sims[q]->cur != (b->cur0[q] ^ b->parity)) return PF_E_INVAL;  // stepped on its own
    for (pf_sim *s : b->sims) {  // fields written since their last fused step: rebuild the liquid maps
        cudaError_t e = ensure_maps<R>(s, b->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(b->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (n < 4 || b->direct_steps < 2 || cs != cudaStreamCaptureStatusNone) {
        int r = batch_step_direct<R>(b, n);
        if (r == PF_OK) b->direct_steps += n;
        return r;
    }
    if (b->parity != 0) {  // the graph starts from the build's buffers
        int r = batch_step_direct<R>(b, 1);
        if (r != PF_OK) return r;
        n -= 1;
    }
    if (!b->graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(e);
        int r = batch_step_direct<R>(b, 2);  // recorded; parity returns to 0
        e = cudaStreamEndCapture(b->stream, &g);
        if (r != PF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return r != PF_OK ? r : cuda_status(e);
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return cuda_status(e);
        }
    }
    for (int q = 0; q + 1 < n; q += 2) {
        cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (n & 1) return batch_step_direct<R>(b, 1);
    return PF_OK;
}

#define PF_BDISPATCH(b, fn, ...) ((b)->precision == PF_FP64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

extern "C" {

int pf_batch_destroy(pf_batch *b)
{
    if (!b) return PF_E_INVAL;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->owns_sims)
        for (pf_sim *s : b->sims)
            if (s) pf_destroy(s);
    dev_free(b->doms, b->stream);
    dev_free(b->items, b->stream);
    dev_free(b->parts, b->stream);
    dev_free(b->counter, b->stream);
    dev_free(b->plan_entries, b->stream);
    dev_free(b->lean_items, b->stream);
    dev_free(b->splits, b->stream);
    dev_free(b->glist, b->stream);
    dev_free(b->plan, b->stream);
    if (b->aux) {
        cudaStreamSynchronize(b->aux);
        cudaStreamDestroy(b->aux);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return PF_OK;
}

int pf_batch_create(int n, const int *nx, const int *ny, const int *nz, const pf_params *params, void *stream,
                    pf_batch **out)
{
    if (!out || n < 1 || !nx || !ny || !nz || !params) return PF_E_INVAL;
    *out = nullptr;
    const int prec = params[0].precision;
    if (prec != PF_FP32 && prec != PF_FP64) return PF_E_INVAL;
    for (int q = 0; q < n; q++)
        if (params[q].precision != prec) return PF_E_INVAL;
    pf_batch *b = new (std::nothrow) pf_batch;
    if (!b) return PF_E_NOMEM;
    b->precision = prec;
    if (stream) {
        b->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete b;
            return cuda_status(e);
        }
        b->own_stream = true;
    }
    for (int q = 0; q < n; q++) {
        pf_sim *s = nullptr;
        int r = pf_create(nx[q], ny[q], nz[q], &params[q], (void *)b->stream, &s);
        if (r != PF_OK) {
            pf_batch_destroy(b);
            return r;
        }
        b->sims.push_back(s);
    }
    *out = b;
    return PF_OK;
}

int pf_batch_domain(pf_batch *b, int d, pf_sim **sim)
{
    if (!b || !sim || d < 0 || d >= (int)b->sims.size()) return PF_E_INVAL;
    *sim = b->sims[d];
    return PF_OK;
}

int pf_batch_init(pf_batch *b, const uint64_t *seeds)
{
    if (!b || !seeds) return PF_E_INVAL;
    for (size_t q = 0; q < b->sims.size(); q++) {
        int r = pf_init(b->sims[q], seeds[q]);
        if (r != PF_OK) return r;
    }
    return PF_OK;
}

int pf_batch_step(pf_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return PF_E_INVAL;
    if (nsteps == 0) return PF_OK;
    return PF_BDISPATCH(b, batch_step, b, nsteps);
}

int pf_batch_sync(pf_batch *b)
{
    if (!b) return PF_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    int first = PF_OK;
    for (pf_sim *s : b->sims) {
        int r = pf_sync(s);
        if (first == PF_OK && r != PF_OK) first = r;
    }
    return first;
}

int pf_batch_set_zchunk(pf_batch *b, int zchunk)
{
    if (!b || zchunk < 0) return PF_E_INVAL;
    if (zchunk != b->zchunk) {
        b->zchunk = zchunk;
        b->built = false;
    }
    return PF_OK;
}

int pf_batch_config(pf_batch *b, int *zchunk, int *general_ctas_per_sm, int *lean_split, int *lean_tile_rows)
{
    if (!b) return PF_E_INVAL;
    if (zchunk) *zchunk = b->zchunk;
    if (general_ctas_per_sm) *general_ctas_per_sm = b->general_per_sm;
    if (lean_split) *lean_split = b->lean_split;
    if (lean_tile_rows) *lean_tile_rows = b->lean_rows;
    return PF_OK;
}

int pf_batch_set_config(pf_batch *b, int zchunk, int general_ctas_per_sm, int lean_split, int lean_tile_rows)
{
    if (!b || zchunk < 0 || (general_ctas_per_sm != 1 && general_ctas_per_sm != 2) ||
        (lean_split != 1 && lean_split != 2 && lean_split != 4) || (lean_tile_rows != 8 && lean_tile_rows != 4))
        return PF_E_INVAL;
    // the next step rebuilds the tables and the graph for the new shape
    b->zchunk = zchunk;
    b->general_per_sm = general_ctas_per_sm;
    b->lean_split = lean_split;
    b->lean_rows = lean_tile_rows;
    b->built = false;
    b->direct_steps = 0;
    return PF_OK;
}

int pf_batch_step_bytes(pf_batch *b, double bytes[2])
{
    if (!b || !bytes) return PF_E_INVAL;
    bytes[0] = bytes[1] = 0.0;
    if (!b->built) return PF_OK;
    std::vector<Partial> h(b->nparts_total);
    cudaError_t e = cudaSuccess;
    if (!h.empty())
        e = cudaMemcpyAsync(h.data(), b->parts.p, h.size() * sizeof(Partial), cudaMemcpyDeviceToHost, b->stream);
    std::vector<LeanStats> ls(b->sims.size());
    for (size_t q = 0; q < b->sims.size() && e == cudaSuccess; q++)
        e = cudaMemcpyAsync(&ls[q], b->sims[q]->lean_stats.p, sizeof(LeanStats), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_status(e);
    for (const Partial &x : h) bytes[0] += x.bytes;
    // the lean kernel's tally of each domain on the lean path (zero for the others)
    if (b->lean_mode)
        for (size_t q = 0; q < ls.size(); q++)
            if (q < b->dom_lean.size() && b->dom_lean[q]) bytes[1] += (double)ls[q].last_bytes;
    return PF_OK;
}

int pf_batch_autotune(pf_batch *b, int trial_steps, int *best, double *best_ms)
{
    if (!b || trial_steps < 2) return PF_E_INVAL;
    const int n = (int)b->sims.size();
    int nzmax = 1;
    for (pf_sim *s : b->sims) nzmax = std::max(nzmax, s->nz);
    // snapshot of every domain's current fields and device state
    std::vector<DevBuf> snap(n);
    std::vector<DevState> ds(n);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    for (int q = 0; q < n && e == cudaSuccess; q++) {
        pf_sim *s = b->sims[q];
        const size_t fb = s->phi[0].bytes + s->mu[0].bytes;
        int r = dev_alloc(snap[q], fb, b->stream);
        if (r != PF_OK) {
            for (auto &x : snap) dev_free(x, b->stream);
            return r;
        }
        e = cudaMemcpyAsync(snap[q].p, s->phi[s->cur].p, s->phi[0].bytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char *)snap[q].p + s->phi[0].bytes, s->mu[s->cur].p, s->mu[0].bytes,
                                cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ds[q], s->state.p, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    std::vector<int> cur(n);
    for (int q = 0; q < n; q++) cur[q] = b->sims[q]->cur;
    auto restore = [&]() -> cudaError_t {
        cudaError_t x = cudaSuccess;
        for (int q = 0; q < n && x == cudaSuccess; q++) {
            pf_sim *s = b->sims[q];
            s->cur = cur[q];
            s->tmap_ok[0] = s->tmap_ok[1] = false;
            x = cudaMemcpyAsync(s->phi[s->cur].p, snap[q].p, s->phi[0].bytes, cudaMemcpyDeviceToDevice, b->stream);
            if (x == cudaSuccess)
                x = cudaMemcpyAsync(s->mu[s->cur].p, (char *)snap[q].p + s->phi[0].bytes, s->mu[0].bytes,
                                    cudaMemcpyDeviceToDevice, b->stream);
            if (x == cudaSuccess) {
                ds[q].shift = 0;  // the snapshot's last shift is in its fields already
                x = cudaMemcpyAsync(s->state.p, &ds[q], sizeof(DevState), cudaMemcpyHostToDevice, b->stream);
            }
            // the plane table of the restored clock and window
            if (x == cudaSuccess && PF_DISPATCH(s, rebuild_table, s, b->stream) != PF_OK) x = cudaErrorLaunchFailure;
        }
        if (x == cudaSuccess) x = cudaStreamSynchronize(b->stream);
        return x;
    };
    // candidates: z-chunk depth x persistent general CTAs per SM (the tile is 32x8 throughout: the
    // liquid maps, the plan and the lean kernel's tensor-map boxes are built per 32x8 tile)
    const int cands[] = {16, 32, 64, 128, 256, 512};
    const int gcands[] = {1, 2};
    const int lcands[] = {1, 2, 4};
    const int rcands[] = {8, 4};
    int bestz = b->zchunk, bestg = b->general_per_sm, bestl = b->lean_split, bestr = b->lean_rows;
    double bestt = 1e300;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int trial = 0; trial < 72; trial++) {
        const int zc = cands[trial / 12], gc = gcands[(trial / 6) % 2], lc = lcands[(trial / 2) % 3],
                  rc = rcands[trial % 2];
        if (e != cudaSuccess) break;
        if (zc > 2 * nzmax && zc != cands[0]) continue;
        b->zchunk = zc;
        b->general_per_sm = gc;
        b->lean_split = lc;
        b->lean_rows = rc;
        b->built = false;
        b->direct_steps = 0;
        int r = PF_BDISPATCH(b, batch_step, b, 1);  // builds the table, warms up
        if (r != PF_OK) break;
        e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) {
            r = PF_BDISPATCH(b, batch_step_direct, b, trial_steps);
            if (r != PF_OK) break;
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms / trial_steps < bestt) {
            bestt = ms / trial_steps;
            bestz = zc;
            bestg = gc;
            bestl = lc;
            bestr = rc;
        }
        if (e == cudaSuccess) e = restore();
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (auto &x : snap) dev_free(x, b->stream);
    b->zchunk = bestz;
    b->general_per_sm = bestg;
    b->lean_split = bestl;
    b->lean_rows = bestr;
    b->built = false;
    b->direct_steps = 0;
    if (e != cudaSuccess) return cuda_status(e);
    if (best) *best = bestz;
    if (best_ms) *best_ms = bestt;
    return PF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// serving loop
// ------------------------------------------------------------------------------------------
namespace {
double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3, REQ_CANCELLED = 4 };

struct ServeReq {
    uint64_t id = 0;
    int nx = 0, ny = 0, nz = 0, nsteps = 0, done_steps = 0;
    pf_params p{};
    uint64_t seed = 0;
    size_t footprint = 0;
    double t_submit = 0.0, t_done = 0.0;
    int state = REQ_QUEUED, status = PF_OK;
    bool cancel = false;
    pf_sim *sim = nullptr;
    double fractions[4] = {0, 0, 0, 0};
    std::vector<float> slab;
};

// device bytes a request holds while it runs: double-buffered FP32 fields plus its small buffers
size_t footprint_of(int nx, int ny, int nz)
{
    const size_t n = (size_t)nx * ny * nz;
    const Geometry g = make_geometry(nx, ny, nz, 0);
    return 2 * n * (16 + 8) + (size_t)2 * nz * 64 + (size_t)2 * g.nparts() * sizeof(Partial) + (size_t)nz * 64 +
           (size_t)2 * nz * g.gx * g.gy + 4096;
}
}  // namespace

struct pf_server {
    size_t budget = 0, used = 0;
    int device = 0, max_active = 256, chunk = 64;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServeReq *> queue;
    std::vector<ServeReq *> running;
    std::unordered_map<uint64_t, ServeReq *> all;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread th;
    pf_batch *batch = nullptr;
    double cell_steps = 0.0, busy = 0.0;
};

// the plane k of a simulation's phi as FP32, component major (4 x nx x ny)
static int read_phi_plane(pf_sim *s, int k, std::vector<float> &out)
{
    const size_t plane = (size_t)s->nx * s->ny;
    DevBuf stg;
    int r = dev_alloc(stg, plane * 4 * sizeof(double), s->stream);
    if (r != PF_OK) return r;
    const KParams<float> kp = make_kparams<float>(s);
    cudaError_t e = launch_pack<float>(kp, (const DevState *)s->state.p, s->phi[s->cur].p, s->mu[s->cur].p,
                                       (double *)stg.p, (double *)nullptr, k, 1, s->stream);
    std::vector<double> h(plane * 4);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), stg.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    dev_free(stg, s->stream);
    if (e != cudaSuccess) return cuda_status(e);
    out.resize(h.size());
    for (size_t q = 0; q < h.size(); q++) out[q] = (float)h[q];
    return PF_OK;
}

static void finish_request(pf_server *v, ServeReq *r)
{
    int st = r->cancel ? PF_E_CANCELLED : pf_sync(r->sim);
    if (st == PF_OK) st = pf_phase_fractions(r->sim, r->fractions);
    double h = 0.0;
    if (st == PF_OK) st = pf_stats(r->sim, nullptr, nullptr, nullptr, &h);
    if (st == PF_OK) {
        int zs = (int)floor(h) - 8;
        zs = std::max(0, std::min(r->nz - 1, zs));
        st = read_phi_plane(r->sim, zs, r->slab);
    }
    pf_destroy(r->sim);
    r->sim = nullptr;
    std::lock_guard<std::mutex> lk(v->mu);
    v->used -= r->footprint;
    r->t_done = now_s();
    r->status = st;
    r->state = r->cancel ? REQ_CANCELLED : (st == PF_OK ? REQ_DONE : REQ_FAILED);
}

static void server_loop(pf_server *v)
{
    cudaSetDevice(v->device);
    for (;;) {
        std::vector<ServeReq *> admit;
        {
            std::unique_lock<std::mutex> lk(v->mu);
            v->cv.wait(lk, [&] { return v->stop || !v->queue.empty() || !v->running.empty(); });
            if (v->stop) break;
            // admission: arrival order; requests behind a waiting one may use only what leaves room for it
            size_t reserve = 0;
            int slots = v->max_active - (int)v->running.size();
            for (auto it = v->queue.begin(); it != v->queue.end() && slots > 0;) {
                ServeReq *r = *it;
                if (r->cancel) {
                    r->state = REQ_CANCELLED;
                    r->status = PF_E_CANCELLED;
                    it = v->queue.erase(it);
                    continue;
                }
                if (v->used + reserve + r->footprint <= v->budget) {
                    v->used += r->footprint;
                    admit.push_back(r);
                    it = v->queue.erase(it);
                    slots--;
                } else {
                    if (reserve == 0) reserve = r->footprint;
                    ++it;
                }
            }
        }
        for (ServeReq *r : admit) {
            pf_sim *sim = nullptr;
            int st = pf_create(r->nx, r->ny, r->nz, &r->p, (void *)v->stream, &sim);
            if (st == PF_OK) pf_set_variant(sim, PF_VARIANT_FUSED);
            if (st == PF_OK) st = pf_init(sim, r->seed);
            std::lock_guard<std::mutex> lk(v->mu);
            if (st != PF_OK) {
                if (sim) pf_destroy(sim);
                v->used -= r->footprint;
                r->status = st;
                r->state = REQ_FAILED;
                r->t_done = now_s();
                continue;
            }
            r->sim = sim;
            r->state = REQ_RUNNING;
            v->running.push_back(r);
            v->batch->built = false;
        }
        if (v->running.empty()) continue;
        // one chunk for every running request: it ends where the next request finishes
        int c = v->chunk;
        for (ServeReq *r : v->running) c = std::min(c, r->nsteps - r->done_steps);
        v->batch->sims.clear();
        for (ServeReq *r : v->running) v->batch->sims.push_back(r->sim);
        const double t0 = now_s();
        int st = c > 0 ? batch_step<float>(v->batch, c) : PF_OK;
        cudaError_t e = cudaStreamSynchronize(v->stream);
        const double t1 = now_s();
        double cells = 0.0;
        for (ServeReq *r : v->running) {
            r->done_steps += c;
            cells += (double)r->nx * r->ny * r->nz;
        }
        std::vector<ServeReq *> keep, done;
        {
            std::lock_guard<std::mutex> lk(v->mu);
            v->cell_steps += cells * c;
            v->busy += t1 - t0;
            for (ServeReq *r : v->running) {
                if (st != PF_OK || e != cudaSuccess || r->cancel || r->done_steps >= r->nsteps)
                    done.push_back(r);
                else
                    keep.push_back(r);
            }
            v->running = keep;
        }
        if (!done.empty()) v->batch->built = false;
        for (ServeReq *r : done) {
            if (st != PF_OK || e != cudaSuccess) r->cancel = false;
            finish_request(v, r);
            if (st != PF_OK && r->status == PF_OK) r->status = st;
        }
        v->cv.notify_all();
    }
    // shutdown: release whatever still runs
    for (ServeReq *r : v->running) {
        r->cancel = true;
        if (r->sim) pf_destroy(r->sim);
        r->sim = nullptr;
        r->state = REQ_CANCELLED;
    }
    v->running.clear();
}

extern "C" {

int pf_server_create(size_t hbm_budget_bytes, int max_active, int chunk, pf_server **out)
{
    if (!out || max_active < 0 || chunk < 0) return PF_E_INVAL;
    *out = nullptr;
    pf_server *v = new (std::nothrow) pf_server;
    if (!v) return PF_E_NOMEM;
    cudaGetDevice(&v->device);
    if (hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete v;
            return PF_E_CUDA;
        }
        hbm_budget_bytes = fr / 10 * 9;
    }
    v->budget = hbm_budget_bytes;
    if (max_active > 0) v->max_active = max_active;
    if (chunk > 0) v->chunk = chunk;
    cudaError_t e = cudaStreamCreateWithFlags(&v->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete v;
        return cuda_status(e);
    }
    v->batch = new (std::nothrow) pf_batch;
    if (!v->batch) {
        cudaStreamDestroy(v->stream);
        delete v;
        return PF_E_NOMEM;
    }
    v->batch->stream = v->stream;
    v->batch->owns_sims = false;
    v->batch->precision = PF_FP32;
    v->th = std::thread(server_loop, v);
    *out = v;
    return PF_OK;
}

int pf_server_destroy(pf_server *v)
{
    if (!v) return PF_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stop = true;
    }
    v->cv.notify_all();
    if (v->th.joinable()) v->th.join();
    v->batch->sims.clear();
    pf_batch_destroy(v->batch);  // does not own the (already released) simulations
    for (auto &kv : v->all) delete kv.second;  // every queued, running or finished record
    v->all.clear();
    v->queue.clear();
    cudaStreamDestroy(v->stream);
    delete v;
    return PF_OK;
}

int pf_submit(pf_server *v, int nx, int ny, int nz, const pf_params *p, uint64_t seed, int nsteps, uint64_t *ticket)
{
    if (!v || !p || !ticket || nx < 1 || ny < 1 || nz < 1 || nsteps < 0) return PF_E_INVAL;
    if (p->precision != PF_FP32 || check_params(p) != PF_OK) return PF_E_INVAL;
    ServeReq *r = new (std::nothrow) ServeReq;
    if (!r) return PF_E_NOMEM;
    r->nx = nx;
    r->ny = ny;
    r->nz = nz;
    r->p = *p;
    r->seed = seed;
    r->nsteps = nsteps;
    r->footprint = footprint_of(nx, ny, nz);
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(v->mu);
        if (r->footprint > v->budget) {
            delete r;
            return PF_E_NOMEM;
        }
        r->id = v->next_id++;
        v->all[r->id] = r;
        v->queue.push_back(r);
        *ticket = r->id;
    }
    v->cv.notify_all();
    return PF_OK;
}

int pf_poll(pf_server *v, uint64_t ticket, double fractions[4], float *slab, double *latency_s)
{
    if (!v) return PF_E_INVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    auto it = v->all.find(ticket);
    if (it == v->all.end()) return PF_E_INVAL;
    ServeReq *r = it->second;
    if (r->state == REQ_QUEUED || r->state == REQ_RUNNING) return PF_E_PENDING;
    int st = r->state == REQ_DONE ? PF_OK : (r->state == REQ_CANCELLED ? PF_E_CANCELLED : r->status);
    if (r->state == REQ_DONE) {
        if (fractions)
            for (int a = 0; a < 4; a++) fractions[a] = r->fractions[a];
        if (slab && !r->slab.empty()) memcpy(slab, r->slab.data(), r->slab.size() * sizeof(float));
    }
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    v->all.erase(it);
    delete r;
    return st;
}

int pf_cancel(pf_server *v, uint64_t ticket)
{
    if (!v) return PF_E_INVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    auto it = v->all.find(ticket);
    if (it == v->all.end()) return PF_E_INVAL;
    it->second->cancel = true;
    return PF_OK;
}

int pf_server_stats(pf_server *v, double *mlups, int *running, int *queued, size_t *used_bytes)
{
    if (!v) return PF_E_INVAL;
    std::lock_guard<std::mutex> lk(v->mu);
    if (mlups) *mlups = v->busy > 0 ? v->cell_steps / v->busy / 1e6 : 0.0;
    if (running) *running = (int)v->running.size();
    if (queued) *queued = (int)v->queue.size();
    if (used_bytes) *used_bytes = v->used;
    return PF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// domain decomposition on one device: slabs with ghost rows (the paper's blocks with ghost layers,
// Section 3.1; Algorithm 1's ghost-layer exchange after each sweep, with Algorithm 2's overlap of the
// mu exchange and the phi-sweep)
// ------------------------------------------------------------------------------------------
struct pf_split {
    int nx = 0, ny = 0, nz = 0, n = 0;
    pf_params p;                       // the domain's parameters (dt resolved)
    std::vector<pf_sim *> slabs;       // slab q: nx x (nys[q] + 2) x nz, own rows 1 .. nys[q]
    std::vector<int> y0, nys;          // first global row and number of own rows of each slab
    std::vector<cudaStream_t> xch;     // the mu ghost exchange of each slab (beside its next phi-sweep)
    std::vector<cudaEvent_t> ev_phi, ev_fin, ev_post, ev_mux;
    cudaEvent_t ev_comb = nullptr;
    DevBuf states;                     // DevState * per slab, the combine kernel's argument
    int latched = PF_OK;
    // a captured graph of two steps (every slab's buffers 0 -> 1 -> 0), replayed on slab 0's stream:
    // its first step forks the other streams off slab 0's, its end joins them back
    cudaGraphExec_t graph = nullptr;
    long long direct_steps = 0;
    cudaEvent_t ev_fork = nullptr, ev_after = nullptr;
};

namespace {
// Row src_row of field src (src_ny rows a plane) into row dst_row of dst (dst_ny rows a plane), in every
// storage plane: one strided copy of nz rows of nx cells.  The slabs shift their rings alike, so a
// storage plane holds the same logical plane in every slab.
cudaError_t copy_row(void *dst, int dst_ny, int dst_row, const void *src, int src_ny, int src_row, int nx, int nz,
                     size_t cell, cudaStream_t st)
{
    const size_t rowb = (size_t)nx * cell;
    return cudaMemcpy2DAsync((char *)dst + (size_t)dst_row * rowb, (size_t)dst_ny * rowb,
                             (const char *)src + (size_t)src_row * rowb, (size_t)src_ny * rowb, rowb, (size_t)nz,
                             cudaMemcpyDeviceToDevice, st);
}

// The ghost rows of slab q from its neighbours' own boundary rows (periodic in y): row 0 takes the
// previous slab's last own row, row nys + 1 the next slab's first own row.
cudaError_t exchange_rows(pf_split *d, int q, int buf, bool phi, cudaStream_t st)
{
    const int P = d->n, qp = (q + P - 1) % P, qn = (q + 1) % P;
    pf_sim *me = d->slabs[q], *pv = d->slabs[qp], *nx_ = d->slabs[qn];
    const size_t w = me->wbytes(), cell = (phi ? 4 : 2) * w;
    void *dst = phi ? me->phi[buf].p : me->mu[buf].p;
    const void *sp = phi ? pv->phi[buf].p : pv->mu[buf].p;
    const void *sn = phi ? nx_->phi[buf].p : nx_->mu[buf].p;
    cudaError_t e = copy_row(dst, me->ny, 0, sp, pv->ny, d->nys[qp], d->nx, d->nz, cell, st);
    if (e == cudaSuccess) e = copy_row(dst, me->ny, d->nys[q] + 1, sn, nx_->ny, 1, d->nx, d->nz, cell, st);
    return e;
}

// nsteps steps of every slab on the slabs' and exchange streams.  in_graph: the steps are being
// captured on slab 0's stream as one graph -- the other streams are forked off it at the start (which
// also orders the first step behind the previous mu exchange) and joined back at the end.
template <typename R>
int split_enqueue(pf_split *d, int nsteps, bool in_graph)
{
    const int P = d->n;
    cudaStream_t s0 = d->slabs[0]->stream;
    if (in_graph) {
        cudaError_t e = cudaEventRecord(d->ev_fork, s0);
        for (int q = 1; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(d->slabs[q]->stream, d->ev_fork, 0);
        for (int q = 0; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(d->xch[q], d->ev_fork, 0);
        if (e != cudaSuccess) return cuda_status(e);
    }
    for (int it = 0; it < nsteps; it++) {
        cudaError_t e = cudaSuccess;
        std::vector<KParams<R>> kp(P);
        for (int q = 0; q < P; q++) kp[q] = make_kparams<R>(d->slabs[q]);
        const int a = d->slabs[0]->cur, b = 1 - a;  // every slab is on the same buffer
        // phi-sweep of every slab: it reads mu^n of its own cells only, so it runs while the mu ghost rows
        // of the previous step are still being copied (Algorithm 2)
        for (int q = 0; q < P && e == cudaSuccess; q++) {
            pf_sim *s = d->slabs[q];
            e = launch_phi_sweep<R>(kp[q], s->geo, s->phi[a].p, s->mu[a].p, s->phi[b].p, (const DevState *)s->state.p,
                                    (const PlaneT<R> *)s->tab.p, s->stream);
            if (e == cudaSuccess) e = cudaEventRecord(d->ev_phi[q], s->stream);
        }
        // phi^{n+1} ghost rows once the neighbours' phi-sweeps are done (Algorithm 1), then the mu-sweep
        // once the mu^n ghost rows have arrived
        for (int q = 0; q < P && e == cudaSuccess; q++) {
            pf_sim *s = d->slabs[q];
            e = cudaStreamWaitEvent(s->stream, d->ev_phi[(q + P - 1) % P], 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, d->ev_phi[(q + 1) % P], 0);
            if (e == cudaSuccess) e = exchange_rows(d, q, b, true, s->stream);
            // (the first step of a graph is ordered behind the last exchange by the fork)
            if (e == cudaSuccess && !(in_graph && it == 0)) e = cudaStreamWaitEvent(s->stream, d->ev_mux[q], 0);
            if (e == cudaSuccess)
                e = launch_mu_sweep<R>(kp[q], s->geo, s->phi[a].p, s->phi[b].p, s->mu[a].p, s->mu[b].p,
                                       (const DevState *)s->state.p, (const PlaneT<R> *)s->tab.p, (Partial *)s->parts.p,
                                       s->stream);
            // the slab's own sums (its finalize runs with the window off)
            if (e == cudaSuccess)
                e = launch_finalize<R>(kp[q], (DevState *)s->state.p, (const Partial *)s->parts.p, s->geo.nparts(),
                                       s->stream);
            if (e == cudaSuccess) e = cudaEventRecord(d->ev_fin[q], s->stream);
        }
        // one window decision on the global interface height, applied to every slab
        for (int q = 1; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s0, d->ev_fin[q], 0);
        if (e == cudaSuccess)
            e = launch_split_combine((DevState *const *)d->states.p, P, d->nx, d->ny, d->nz,
                                     d->p.window_trigger_z > 0.0 ? 1 : 0, d->p.window_trigger_z, s0);
        if (e == cudaSuccess) e = cudaEventRecord(d->ev_comb, s0);
        for (int q = 0; q < P && e == cudaSuccess; q++) {
            pf_sim *s = d->slabs[q];
            if (q > 0) e = cudaStreamWaitEvent(s->stream, d->ev_comb, 0);
            if (e == cudaSuccess)
                e = launch_post<R>(kp[q], (const DevState *)s->state.p, s->phi[b].p, s->mu[b].p, (PlaneT<R> *)s->tab.p,
                                   s->stream);
            if (e == cudaSuccess) e = cudaEventRecord(d->ev_post[q], s->stream);
        }
        // mu^{n+1} ghost rows after every neighbour's post (its window fill included), on the exchange
        // streams: they overlap the next phi-sweep, and the next mu-sweep waits for them
        for (int q = 0; q < P && e == cudaSuccess; q++) {
            e = cudaStreamWaitEvent(d->xch[q], d->ev_post[(q + P - 1) % P], 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(d->xch[q], d->ev_post[q], 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(d->xch[q], d->ev_post[(q + 1) % P], 0);
            if (e == cudaSuccess) e = exchange_rows(d, q, b, false, d->xch[q]);
            if (e == cudaSuccess) e = cudaEventRecord(d->ev_mux[q], d->xch[q]);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (d->latched == PF_OK) d->latched = cuda_status(e);
            return d->latched;
        }
        for (pf_sim *s : d->slabs) {
            s->cur = b;
            s->tmap_ok[0] = s->tmap_ok[1] = false;
            s->last_kind = 0;
        }
    }
    if (in_graph) {  // join: slab 0's stream waits for every other stream's last work
        cudaError_t e = cudaSuccess;
        for (int q = 1; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s0, d->ev_post[q], 0);
        for (int q = 0; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s0, d->ev_mux[q], 0);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return PF_OK;
}

// pf_split_step's driver: the first steps and short calls launch directly; otherwise a captured graph of
// two steps is replayed (the slabs' launches and copies are paid once).  Work launched directly before a
// replay is gathered onto slab 0's stream first, and the other streams wait for the replays before
// their next direct work (events recorded inside a graph do not order work outside it).
template <typename R>
int split_step(pf_split *d, int nsteps)
{
    const int P = d->n;
    cudaStream_t s0 = d->slabs[0]->stream;
    auto fail = [&](cudaError_t e) {
        cudaGetLastError();
        if (d->latched == PF_OK) d->latched = cuda_status(e);
        return d->latched;
    };
    if (nsteps < 4 || d->direct_steps < 2) {
        const int r = split_enqueue<R>(d, nsteps, false);
        if (r == PF_OK) d->direct_steps += nsteps;
        return r == PF_OK ? r : (d->latched = d->latched == PF_OK ? r : d->latched);
    }
    if (d->slabs[0]->cur != 0) {  // the graph starts from buffer 0
        const int r = split_enqueue<R>(d, 1, false);
        if (r != PF_OK) return d->latched = d->latched == PF_OK ? r : d->latched;
        nsteps -= 1;
    }
    cudaError_t e = cudaSuccess;
    if (!d->graph) {
        // ordered behind the direct steps (the capture starts on slab 0's stream)
        for (int q = 1; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s0, d->ev_post[q], 0);
        for (int q = 0; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s0, d->ev_mux[q], 0);
        if (e != cudaSuccess) return fail(e);
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(e);
        const int r = split_enqueue<R>(d, 2, true);  // recorded, not run: buffers end where they started
        e = cudaStreamEndCapture(s0, &g);
        if (r != PF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(e != cudaSuccess ? e : cudaErrorUnknown);
        }
        e = cudaGraphInstantiate(&d->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            d->graph = nullptr;
            return fail(e);
        }
    } else {
        // the direct work since the last replay, gathered onto slab 0's stream (after a capture the
        // events' last records are the capture's, which no work outside it may wait on: the gather
        // before the capture stands for them)
        for (int q = 1; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s0, d->ev_post[q], 0);
        for (int q = 0; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(s0, d->ev_mux[q], 0);
    }
    for (int q = 0; q + 1 < nsteps && e == cudaSuccess; q += 2) e = cudaGraphLaunch(d->graph, s0);
    // the other streams' next direct work after the replays
    if (e == cudaSuccess) e = cudaEventRecord(d->ev_after, s0);
    for (int q = 1; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(d->slabs[q]->stream, d->ev_after, 0);
    for (int q = 0; q < P && e == cudaSuccess; q++) e = cudaStreamWaitEvent(d->xch[q], d->ev_after, 0);
    if (e != cudaSuccess) return fail(e);
    // the exchange events' next use is a direct step: they must describe the replayed steps' end
    for (int q = 0; q < P && e == cudaSuccess; q++) e = cudaEventRecord(d->ev_mux[q], d->xch[q]);
    for (int q = 0; q < P && e == cudaSuccess; q++) e = cudaEventRecord(d->ev_post[q], d->slabs[q]->stream);
    if (e != cudaSuccess) return fail(e);
    if (nsteps & 1) {
        const int r = split_enqueue<R>(d, 1, false);
        if (r != PF_OK) return d->latched = d->latched == PF_OK ? r : d->latched;
    }
    return PF_OK;
}
}  // namespace

extern "C" {

int pf_split_destroy(pf_split *d)
{
    if (!d) return PF_E_INVAL;
    for (cudaStream_t x : d->xch)
        if (x) cudaStreamSynchronize(x);
    for (pf_sim *s : d->slabs)
        if (s) pf_destroy(s);
    for (cudaStream_t x : d->xch)
        if (x) cudaStreamDestroy(x);
    for (auto *v : {&d->ev_phi, &d->ev_fin, &d->ev_post, &d->ev_mux})
        for (cudaEvent_t ev : *v)
            if (ev) cudaEventDestroy(ev);
    if (d->ev_comb) cudaEventDestroy(d->ev_comb);
    if (d->ev_fork) cudaEventDestroy(d->ev_fork);
    if (d->ev_after) cudaEventDestroy(d->ev_after);
    if (d->graph) cudaGraphExecDestroy(d->graph);
    dev_free(d->states, nullptr);
    delete d;
    return PF_OK;
}

int pf_split_create(int nx, int ny, int nz, const pf_params *p, int nslabs, pf_split **out)
{
    if (!out) return PF_E_INVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nslabs < 1 || nslabs > ny) return PF_E_INVAL;
    int r = check_params(p);
    if (r != PF_OK) return r;
    if (p->precision == PF_FP32_COMP) return PF_E_INVAL;
    pf_split *d = new (std::nothrow) pf_split;
    if (!d) return PF_E_NOMEM;
    d->nx = nx;
    d->ny = ny;
    d->nz = nz;
    d->n = nslabs;
    d->p = *p;
    if (!(d->p.dt > 0.0)) d->p.dt = default_dt(d->p, nz);
    pf_params q = d->p;
    q.window_trigger_z = 0.0;  // the slabs never move their windows on their own: the combine kernel does
    for (int k = 0; k < nslabs && r == PF_OK; k++) {
        const int y0 = (int)((long long)k * ny / nslabs), y1 = (int)((long long)(k + 1) * ny / nslabs);
        d->y0.push_back(y0);
        d->nys.push_back(y1 - y0);
        pf_sim *s = nullptr;
        r = pf_create(nx, y1 - y0 + 2, nz, &q, nullptr, &s);
        if (r != PF_OK) break;
        d->slabs.push_back(s);
        s->variant = PF_VARIANT_UNFUSED;  // Algorithm 1's two sweeps
        s->gy0 = y0 - 1;                  // local row 0 is the ghost row below the slab
        s->gny = ny;
        s->red_j0 = 1;
        s->red_j1 = y1 - y0 + 1;
        cudaStream_t x = nullptr;
        cudaEvent_t e4[4] = {nullptr, nullptr, nullptr, nullptr};
        cudaError_t e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        for (int j = 0; j < 4 && e == cudaSuccess; j++) e = cudaEventCreateWithFlags(&e4[j], cudaEventDisableTiming);
        d->xch.push_back(x);
        d->ev_phi.push_back(e4[0]);
        d->ev_fin.push_back(e4[1]);
        d->ev_post.push_back(e4[2]);
        d->ev_mux.push_back(e4[3]);
        if (e != cudaSuccess) r = cuda_status(e);
    }
    if (r == PF_OK) {
        cudaError_t e = cudaEventCreateWithFlags(&d->ev_comb, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d->ev_after, cudaEventDisableTiming);
        if (e != cudaSuccess) r = cuda_status(e);
    }
    if (r == PF_OK) r = dev_alloc(d->states, sizeof(DevState *) * nslabs, nullptr);
    if (r == PF_OK) {
        std::vector<DevState *> ptr;
        for (pf_sim *s : d->slabs) ptr.push_back((DevState *)s->state.p);
        cudaError_t e = cudaMemcpy(d->states.p, ptr.data(), sizeof(DevState *) * nslabs, cudaMemcpyHostToDevice);
        // the exchange events start recorded (an initial state has valid ghost rows)
        for (int k = 0; k < nslabs && e == cudaSuccess; k++) e = cudaEventRecord(d->ev_mux[k], d->xch[k]);
        if (e != cudaSuccess) r = cuda_status(e);
    }
    if (r != PF_OK) {
        pf_split_destroy(d);
        return r;
    }
    *out = d;
    return PF_OK;
}

int pf_split_sync(pf_split *d)
{
    if (!d) return PF_E_INVAL;
    int r = d->latched;
    d->latched = PF_OK;
    for (cudaStream_t x : d->xch)
        if (cudaStreamSynchronize(x) != cudaSuccess && r == PF_OK) r = PF_E_CUDA;
    for (pf_sim *s : d->slabs) {
        const int rs = pf_sync(s);
        if (r == PF_OK) r = rs;
    }
    return r;
}

int pf_split_init(pf_split *d, uint64_t seed)
{
    if (!d) return PF_E_INVAL;
    int r = pf_split_sync(d);
    (void)r;
    // every slab, its ghost rows included, takes the rows of the global domain it covers
    for (pf_sim *s : d->slabs) {
        const int ri = pf_init(s, seed);
        if (ri != PF_OK) return ri;
    }
    return PF_OK;
}

int pf_split_step(pf_split *d, int nsteps)
{
    if (!d || nsteps < 0) return PF_E_INVAL;
    if (d->latched != PF_OK) return d->latched;
    return d->p.precision == PF_FP64 ? split_step<double>(d, nsteps) : split_step<float>(d, nsteps);
}

int pf_split_read_fields(pf_split *d, double *phi, double *mu, size_t cap_cells)
{
    if (!d || cap_cells < (size_t)d->nx * d->ny * d->nz) return PF_E_INVAL;
    int r = pf_split_sync(d);
    if (r != PF_OK) return r;
    const size_t nxy = (size_t)d->nx, plane = (size_t)d->nx * d->ny, n = plane * d->nz;
    for (int q = 0; q < d->n; q++) {
        pf_sim *s = d->slabs[q];
        const size_t sn = s->ncell(), splane = (size_t)d->nx * s->ny;
        std::vector<double> tp(phi ? 4 * sn : 0), tm(mu ? 2 * sn : 0);
        r = pf_read_fields(s, phi ? tp.data() : nullptr, mu ? tm.data() : nullptr, sn);
        if (r != PF_OK) return r;
        // the slab's own rows 1 .. nys into global rows y0 ..
        for (int k = 0; k < d->nz; k++)
            for (int j = 0; j < d->nys[q]; j++) {
                const size_t gsrc = (size_t)k * splane + (size_t)(j + 1) * nxy;
                const size_t gdst = (size_t)k * plane + (size_t)(d->y0[q] + j) * nxy;
                for (int c = 0; c < 4 && phi; c++)
                    memcpy(phi + c * n + gdst, tp.data() + c * sn + gsrc, nxy * sizeof(double));
                for (int c = 0; c < 2 && mu; c++)
                    memcpy(mu + c * n + gdst, tm.data() + c * sn + gsrc, nxy * sizeof(double));
            }
    }
    return PF_OK;
}

int pf_split_stats(pf_split *d, double *t, double *window_offset, double *h_int, int *planes_shifted)
{
    if (!d) return PF_E_INVAL;
    int r = pf_split_sync(d);
    if (r != PF_OK) return r;
    DevState ds;
    r = read_state(d->slabs[0], &ds);
    if (r != PF_OK) return r;
    if (t) *t = ds.t;
    if (window_offset) *window_offset = ds.off;
    if (planes_shifted) *planes_shifted = ds.nshift_total;
    if (h_int) {
        // of the current fields: each slab's FP64 sum over its own rows
        double liq = 0.0;
        for (pf_sim *s : d->slabs) {
            double acc[8];
            r = PF_DISPATCH(s, do_reduce, s, acc);
            if (r != PF_OK) return r;
            liq += acc[6];
        }
        *h_int = liq / ((double)d->nx * (double)d->ny);
    }
    return PF_OK;
}

}  // extern "C"
