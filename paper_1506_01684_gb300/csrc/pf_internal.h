// pf_internal.h -- structures and launcher declarations shared by the host runtime and the
// CUDA kernels of the phase-field time step.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/pf.h"

namespace pf {

// Device-resident state of one simulation.  Kernels read the time, window offset and the
// ring-buffer base from here, so a sequence of steps needs no host round trip and can be
// replayed from a captured graph.  Written by finalize_kernel (one thread) and the host.
struct DevState {
    double t;          // simulation time of the current source fields
    double off;        // window offset in planes (FP64, integer valued)
    double h_int;      // interface height measured after the last step
    int zbase;         // storage plane of logical plane 0 (moving-window ring buffer)
    int shift;         // planes shifted by the last finalize (0: none); read by post_kernel
    int nonfinite;     // sticky: 1 a non-finite value was seen, 2 a bounded device wait gave up
    int nshift_total;  // planes shifted since init
    double liq;        // sum over the counted cells of (1 - phi_l) measured after the last step (FP64)
};

// Per-CTA partial sums written by the mu-sweep epilogue (FP64).
struct Partial {
    double liq_deficit;  // sum over the CTA's cells of (1 - phi_l^{n+1})
    double nonfinite;    // > 0 when a cell of the CTA produced a non-finite value
    double bytes;        // algorithmic HBM bytes of the step for the CTA's cells (compulsory
                         // loads and stores of the design that ran; read back for the roofline)
    double timeout;      // > 0 when a bounded wait of the CTA gave up
};

// Per-simulation statistics of the lean kernel (the fused step's pure-liquid planes), summed
// atomically by its CTAs and folded into the step's state by finalize.
struct LeanStats {
    unsigned long long bytes;       // algorithmic bytes of the current step
    int nonfinite;                  // a non-finite mu^{n+1} was produced
    int timeout;                    // a bounded wait gave up
    unsigned long long last_bytes;  // bytes of the last finished step (read by the host)
    unsigned gcount, gnext;         // (tile, chunk) items with general planes; next one to take
    unsigned gnext_mu;              // next item of the general planes' mu-sweep
    int map_changed;                // a liquid-map entry of the new field differs from the source's
    int plan_valid;                 // the plan (splits, item list, zeroed partials) describes the
                                    // current source field: the next plan kernel has nothing to do
    int pad_;
};

// Temperature-dependent constants of one x-y plane (cell centres) or one z-face level,
// formed once per plane in FP64 and rounded to the stencil precision (the per-slice
// precompute of the paper's Section 3.3).  16 words so that it stages with vector loads.
template <typename R>
struct PlaneT {
    R T, epsT, Toeps, pad0;
    R chat[4][2];  // cE_a + kT_a (T - TE)
    R sT[4];       // s_a (T - TE)
};

// Scalar parameters handed to the kernels by value.  R is the stencil precision.
template <typename R>
struct KParams {
    int nx, ny, nz;
    int zchunk;  // planes per CTA along z
    int window;  // 1: moving window enabled
    int tgx, tgy;  // tile grid of the fused step (liquid map layout)
    int test_flags;  // bit 0: the lean kernel's producer withholds its copies (tests of the bounded waits)
    // a slab of a decomposed domain (pf_split): local row j is global row (j + gy0) mod gny of a domain
    // gny rows high (gny = 0: the domain itself); rows [red_j0, red_j1) are the slab's own rows, the only
    // ones the reductions count (the others are ghost rows)
    int gy0, gny, red_j0, red_j1;
    R dx, inv_dx, inv_2dx, inv_4dx;
    R eps, inv_eps;
    R c_phi;  // dt / (tau eps)
    R dt, inv_dt;
    R gamma2[6], gamma3[4];
    R inv2A[4];  // 1/(2 A_a)
    R inv4A[4];  // 1/(4 A_a)
    R DinvA[4];  // D_a/(2 A_a)
    R kT[4][2];
    R at_pref;   // pi eps / 4
    R grad_thr;  // 1e-20 / dx^2
    R obst;      // 16 / pi^2
    R dTstep;    // -G v dt
    // FP64 data for the plane table, the reductions and the clock
    double T0, G, v, TE, dx64, dt64, eps64, window_trigger_z;
    double cE[4][2], kT64[4][2], s64[4], A64[4];
    // general parabolic thermodynamics (matrix curvatures A_a, pair relaxation times)
    int gen;          // 1: K_a = (1/2) A_a^{-1} is a full 2x2 matrix; 0: K_a = inv2A[a] times the identity
    int gen_tau;      // 1: tau interpolated over the phase pairs at the cell's phi^n
    R K[4][3];        // K_a: (K11, K12, K22)
    R DK[4][3];       // D_a K_a
    R psiK[4][3];     // (K11/2, K12, K22/2): (1/2) mu . K_a mu = psiK0 mu0^2 + psiK1 mu0 mu1 + psiK2 mu1^2
    R tau_ab[6];      // pairs 01 02 03 12 13 23
    R dt_eps;         // dt / eps
    R liqC1, liqC0[2];  // pure-liquid update mu + C1 (7-point Laplacian sum) + C0 with matrix curvatures
    double K64[4][3];   // K_a in FP64 (reductions)
};

// The lean kernel's tensor maps of one mu buffer, all over the same 3D tensor (2 nx words, ny rows,
// nz storage planes): the tile box with its one-cell halo (TX + 4 cells x TY + 2 rows), the box of the
// periodic x images (2 cells x TY rows: the wrapped column at x = -1 or x = nx) and the box of the
// periodic y images (TX + 4 cells x 1 row: the wrapped row at y = -1 or y = ny).
struct alignas(64) LeanMaps {
    CUtensorMap box, ximg, yimg;
};

// One domain of a batched step: its parameters, ping-pong field buffers, state, plane table and
// partial sums, and its fused-step tile grid; for the lean path also the TMA tensor maps of its mu
// buffers, its plan (splits per (tile, chunk)) and its lean statistics.
template <typename R>
struct alignas(128) BatchDomain {  // the alignment of its tensor maps
    LeanMaps mu_map[2];      // TMA maps of mu[0], mu[1] (lean path)
    KParams<R> kp;
    void *phi[2], *mu[2];
    unsigned char *tmap[2];  // liquid maps of the two field buffers
    DevState *st;
    PlaneT<R> *tab;
    Partial *parts;
    int2 *splits;            // the step's lean / general split per (tile, chunk) (lean path)
    LeanStats *lean;         // the domain's lean statistics (lean path)
    int gx, gy, gz, nsub;    // fused-step tile grid; lean CTAs per z chunk
};
// The general-plane list of a batched step: (domain, item) pairs and their counters.
struct BatchPlan {
    unsigned gcount, gnext, gnext_mu, pad_;
};
// One work item of a batched step: a tile of one domain.
struct BatchItem {
    int dom, bx, by, bz;
};

// Most work units an item of the general planes is cut into (the general planes' sweeps, pf_kernels.cuh).
#ifndef PF_MAX_UNITS
#define PF_MAX_UNITS 8
#endif
constexpr int kMaxUnits = PF_MAX_UNITS;

// Launch geometry of the sweep kernels.
struct Geometry {
    int tx, ty;     // CTA tile in x and y (columns)
    int zchunk;     // planes per CTA
    int gx, gy, gz; // grid
    int nparts() const { return gx * gy * gz; }
};

Geometry make_geometry(int nx, int ny, int nz, int zchunk_hint);

// Parameter plumbing shared with the allocation-free entry point (pf_noalloc.cu).
template <typename R>
KParams<R> kparams_for(const pf_params &p, int nx, int ny, int nz, const Geometry &g);
double resolved_dt(const pf_params &p, int nz);
int validate_params(const pf_params *p);

// Launchers (defined in pf_kernels.cuh, instantiated for float and double).  pdl: launch with
// programmatic stream serialisation (the kernel may be scheduled while the one ahead of it in the stream
// is still running and waits for it on the device before it depends on its results).
template <typename R>
cudaError_t launch_phi_sweep(const KParams<R> &kp, const Geometry &g, const void *phi, const void *mu,
                             void *phi_out, const DevState *st, const PlaneT<R> *tab, cudaStream_t s);
template <typename R>
cudaError_t launch_mu_sweep(const KParams<R> &kp, const Geometry &g, const void *phi_old, const void *phi_new,
                            const void *mu, void *mu_out, const DevState *st, const PlaneT<R> *tab,
                            Partial *parts, cudaStream_t s);
// tmap_in / tmap_out: the liquid maps (one byte per storage plane and tile of the fused grid:
// 1 = every cell of the tile in that plane is exactly pure liquid) of the source and the new
// fields; nullptr disables the lean path.
template <typename R>
cudaError_t launch_fused_step(const KParams<R> &kp, const Geometry &g, const void *phi, const void *mu,
                              void *phi_out, void *mu_out, const DevState *st, const PlaneT<R> *tab, Partial *parts,
                              cudaStream_t s, const unsigned char *tmap_in = nullptr,
                              unsigned char *tmap_out = nullptr, bool lean_here = true);
// The pure-liquid planes of the fused step (lean_step_kernel), launched beside the fused kernel
// run with lean_here = 0: grid (tgx, tgy, gz * nsub), one CTA per tile and sub-chunk of a z chunk.
// mu_map: the LeanMaps of the source mu buffer (3D: 2 nx words, ny, nz); stats: the sim's lean
// statistics (folded in by the next finalize).  Returns cudaErrorInvalidValue when the map layout
// or the chunking does not fit the kernel.
template <typename R>
cudaError_t launch_lean_step(const KParams<R> &kp, const Geometry &g, int nsub, const void *mu_map, const void *mu,
                             void *phi_out, void *mu_out, const DevState *st, LeanStats *stats, cudaStream_t s,
                             const unsigned char *tmap_in, unsigned char *tmap_out, const int2 *splits,
                             bool pdl = false, const void *mu_lo = nullptr, void *phi_out_lo = nullptr,
                             void *mu_out_lo = nullptr);  // compensated FP32: the low words
// Plan of a fused step with the lean kernel (plan_kernel): each (tile, chunk) item's split into
// lean and general planes (splits, gx*gy*gz), the list of items with general planes (glist,
// count in stats->gcount; finalize resets the counters), zeroed partials for the all-lean items.
template <typename R>
cudaError_t launch_plan(const KParams<R> &kp, const Geometry &g, const DevState *st, const unsigned char *tmap_in,
                        int2 *splits, int *glist, LeanStats *stats, Partial *parts, cudaStream_t s, bool pdl = false);
// The general planes of the listed items: ctas persistent CTAs (general_step_kernel).
template <typename R>
cudaError_t launch_general_step(const KParams<R> &kp, const void *phi, const void *mu, void *phi_out, void *mu_out,
                                const DevState *st, const PlaneT<R> *tab, Partial *parts,
                                const unsigned char *tmap_in, unsigned char *tmap_out, const int2 *splits,
                                const int *glist, LeanStats *stats, int ctas, cudaStream_t s);
template <typename R>
int general_ctas_per_sm();
// The general planes of the listed items as Algorithm 1's two sweeps: the phi-sweep (phi^{n+1} and
// its liquid-map entries) and then the mu-sweep (phi^{n+1} of lean tile planes taken as e_l), each
// by persistent CTAs over the list; the mu partials carry both sweeps' bytes (22 words a cell).
// Each listed item's general range is cut into U units (U from the list length and the persistent CTA
// count, the same in both sweeps); with U > 1 each unit's mu-sweep partial goes to subparts (kMaxUnits
// slots per item) and the item's last unit to finish sums them in unit order into parts[item] (subcnt:
// one counter per item, zero between steps).
template <typename R>
cudaError_t launch_general_sweeps(const KParams<R> &kp, const void *phi, const void *mu, void *phi_out, void *mu_out,
                                  const DevState *st, const PlaneT<R> *tab, Partial *parts,
                                  const unsigned char *tmap_in, unsigned char *tmap_out,
                                  const int2 *splits, const int *glist, LeanStats *stats, int phi_ctas, int mu_ctas,
                                  cudaStream_t s, Partial *subparts, unsigned *subcnt, bool pdl = false,
                                  bool after_lean = false,  // after_lean: launched right behind the lean kernel
                                  const void *phi_lo = nullptr, void *phi_out_lo = nullptr,  // compensated FP32:
                                  const void *mu_lo = nullptr, void *mu_out_lo = nullptr,    // the low words
                                  bool prio = false);  // prio: the device's highest launch priority
template <typename R>
void general_sweep_ctas_per_sm(int *phi_per_sm, int *mu_per_sm);
// liquid map of a field (for states not produced by a fused step)
template <typename R>
cudaError_t launch_classify(const KParams<R> &kp, const DevState *st, const void *phi, unsigned char *tmap,
                            cudaStream_t s, const void *phi_lo = nullptr);  // phi_lo: compensated low words
template <typename R>
cudaError_t launch_finalize(const KParams<R> &kp, DevState *st, const Partial *parts, int nparts, cudaStream_t s,
                            LeanStats *lean = nullptr, bool pdl = false);
// Batched fused step of ndoms domains: counter reset, persistent kernel (ctas CTAs) over the
// work items, per-domain finalize and post.  parity: index of the source buffers.
template <typename R>
cudaError_t launch_batched_step(const BatchDomain<R> *doms, int ndoms, const BatchItem *items, int nitems,
                                unsigned *counter, int parity, int ctas, int post_blocks, cudaStream_t s);
template <typename R>
int fused_ctas_per_sm();
// Batched step on the lean path: counters reset, plan over the (domain, item) entries, the general
// planes' two sweeps (persistent CTAs over the batch-wide list), the lean kernel over its items
// (domain, tile x, row block y, chunk * nsub + sub) with lean_rows-row CTA tiles (8: a whole map tile,
// 4: half of one; the domains' tensor maps must have the matching boxes); domains without TMA maps
// run the fused tile over their items (fitems); then per-domain finalize and post.  parity: index of
// the source buffers.  sym: every domain has the symmetric parameter set; aux: the general sweeps
// run on it beside the lean kernel.
template <typename R>
cudaError_t launch_batched_lean_step(const BatchDomain<R> *doms, int ndoms, const int2 *plan_entries, int nplan,
                                     const int4 *lean_items, int nlean, int2 *glist, BatchPlan *plan,
                                     int phi_ctas, int mu_ctas, const BatchItem *fitems, int nfitems,
                                     unsigned *counter, int fctas, int parity, int post_blocks, cudaStream_t s,
                                     bool sym, cudaStream_t aux = nullptr, cudaEvent_t fork = nullptr,
                                     cudaEvent_t join = nullptr, int lean_rows = 8);
template <typename R>
void batched_general_ctas_per_sm(int *phi_per_sm, int *mu_per_sm);
// The window decision of a decomposed domain (one thread): the global interface height from the slabs'
// liquid-deficit sums (in slab order) over nx * ny_global cells, then the same shift applied to every
// slab's state (each slab's finalize ran with the window off).
cudaError_t launch_split_combine(DevState *const *states, int nslabs, int nx, int ny_global, int nz, int window,
                                 double trigger, cudaStream_t s);
template <typename R>
cudaError_t launch_post(const KParams<R> &kp, const DevState *st, void *phi, void *mu, PlaneT<R> *tab,
                        cudaStream_t s, void *phi_lo = nullptr, void *mu_lo = nullptr,
                        unsigned char *tmap = nullptr, bool pdl = false);
template <typename R>
cudaError_t launch_init(const KParams<R> &kp, void *phi, void *mu, const double *seeds, int n_grains, int H,
                        cudaStream_t s);
template <typename R>
cudaError_t launch_reduce(const KParams<R> &kp, const DevState *st, const void *phi, const void *mu,
                          double *plane_sums /* nz x 8 */, cudaStream_t s, const void *phi_lo = nullptr,
                          const void *mu_lo = nullptr);
// AoS fields <-> SoA staging of host element type H (double or float) for logical planes [k0, k0 + nk)
template <typename R, typename H>
cudaError_t launch_pack(const KParams<R> &kp, const DevState *st, const void *phi, const void *mu, H *phi_soa,
                        H *mu_soa, int k0, int nk, cudaStream_t s, const void *phi_lo = nullptr,
                        const void *mu_lo = nullptr);
template <typename R, typename H>
cudaError_t launch_unpack(const KParams<R> &kp, const DevState *st, void *phi, void *mu, const H *phi_soa,
                          const H *mu_soa, int k0, int nk, cudaStream_t s, void *phi_lo = nullptr,
                          void *mu_lo = nullptr);
// Interface mesh of phase `phase` (marching tetrahedra over the cell centres), in segments of up to
// 256 cubes of one row of one layer, ordered (k ny + j) nb + b with nb = ceil(nx / 256): triangles
// per segment; the offsets and ids of the non-empty segments with the totals (triangles, non-empty
// segments; one CTA; counts padded with zeros to nseg_pad, a multiple of 16); the triangles of the
// listed segments (9 floats a triangle).
template <typename R>
cudaError_t launch_mesh_count(const KParams<R> &kp, const DevState *st, const void *phi, int phase, double iso,
                              unsigned *seg_counts, cudaStream_t s);
template <typename R>
cudaError_t launch_mesh_scan(const unsigned *seg_counts, size_t nseg_pad, unsigned *ne_seg, unsigned long long *ne_off,
                             unsigned long long *totals, cudaStream_t s);
template <typename R>
cudaError_t launch_mesh_emit(const KParams<R> &kp, const DevState *st, const void *phi, int phase, double iso,
                             const unsigned *ne_seg, const unsigned long long *ne_off, unsigned n_ne,
                             unsigned long long ntris, float *tris, cudaStream_t s);

// Compensated FP32 (state = hi + lo) variants of the two sweeps.
cudaError_t launch_phi_sweep_comp(const KParams<float> &kp, const Geometry &g, const void *phi, const void *phi_lo,
                                  const void *mu, void *phi_out, void *phi_out_lo, const DevState *st,
                                  const PlaneT<float> *tab, cudaStream_t s);
cudaError_t launch_mu_sweep_comp(const KParams<float> &kp, const Geometry &g, const void *phi_old,
                                 const void *phi_new, const void *mu, const void *mu_lo, void *mu_out,
                                 void *mu_out_lo, const DevState *st, const PlaneT<float> *tab, Partial *parts,
                                 cudaStream_t s);

}  // namespace pf
