/*
 * pf.h -- C ABI of the GB300 (sm_103a) library for the explicit time step of the
 * grand-potential phase-field model of ternary eutectic directional solidification
 * (Bauer et al., arXiv:1506.01684).
 *
 * Model (paper Section 2): four phase fields phi_a (a = 0,1,2 solid, 3 liquid) on the
 * Gibbs simplex and two chemical potentials mu (K = 3 components), evolved by Eq. 1-2
 * (phi) and Eq. 3-4 (mu, with the anti-trapping current) under the frozen temperature
 * T = T0 + G (z - v t), with a moving window along z.  One time step is Algorithm 1:
 * phi-sweep, then mu-sweep reading phi at both time levels.
 *
 * Conventions shared by every entry point:
 *   - Grid: nx * ny * nz cells, cell (i,j,k), x fastest; periodic in x and y,
 *     zero-gradient (mirror) in z; cell centres at z = (k + window_offset) * dx.
 *   - Host field layout (read/write calls): FP64, structure of arrays
 *     [component][z][y][x]; phi has 4 components, mu has 2.
 *   - Ownership: the library owns every device buffer and handle it creates; the
 *     caller owns every host buffer it passes and keeps it alive for the call.
 *   - Errors: every call returns a status (PF_OK or a negative PF_E_*); nothing
 *     throws or aborts across the ABI.  Device work is asynchronous on the
 *     simulation's stream; device-side errors (non-finite values, CUDA faults) are
 *     latched and returned by the next synchronising call.
 *   - Threads: a pf_sim is used by one thread at a time; a pf_server is internally
 *     synchronised.
 */
#ifndef PF_GB300_H
#define PF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
    PF_OK = 0,
    PF_E_INVAL = -1,     /* invalid argument (null pointer, size, parameter) */
    PF_E_NOMEM = -2,     /* device or host allocation failed / admission refused */
    PF_E_CUDA = -3,      /* a CUDA call failed */
    PF_E_UNSTABLE = -4,  /* a non-finite value appeared in phi or mu */
    PF_E_TIMEOUT = -5,   /* a bounded wait gave up */
    PF_E_CANCELLED = -6, /* a served request was cancelled */
    PF_E_PENDING = 1     /* pf_poll only: the request is not finished yet */
};

/* arithmetic of the stencil kernels and the field storage */
enum {
    PF_FP64 = 0,     /* FP64 storage and arithmetic (the plain reference path) */
    PF_FP32 = 1,     /* FP32 storage and arithmetic */
    PF_FP32_COMP = 2 /* FP32 arithmetic, state kept as FP32 high + FP32 low words (compensated) */
};

#define PF_PARAMS_VERSION 2

/*
 * Physical and numerical parameters, always FP64 (the library converts them to the
 * kernel precision).  Readings of the paper where it prints no value (parabolic Gibbs
 * energies f_a(c,T) = c . A_a c + B_a(T) . c + C_a(T) as grand potentials, Section 2):
 *   psi_a(mu,T) = -(1/2) mu . K_a mu - mu . chat_a(T) + s_a (T - TE),  K_a = (1/2) A_a^{-1},
 *   chat_a(T) = cE_a + kT_a (T - TE),  c^a = K_a mu + chat_a(T),
 *   A_a = A[a] times the identity, or the symmetric matrix Am[a] when Am[a][0] > 0,
 *   chi = sum_a h_a K_a,  mu^{n+1} = mu^n + chi^{-1} (source)  (2x2),
 *   h_a = phi_a^2 / sum phi_b^2,  g_a = phi_a,  M = sum_a D_a h_a K_a,
 *   tau(phi) = sum_{a<b} tau_ab phi_a phi_b / sum_{a<b} phi_a phi_b at phi^n (tau on a
 *     single-phase cell) when tau_ab is set, else tau,
 *   a = sum_{a<b} gamma2_ab |phi_a grad phi_b - phi_b grad phi_a|^2,
 *   omega = (16/pi^2) sum gamma2_ab phi_a phi_b + sum gamma3_abd phi_a phi_b phi_d.
 */
typedef struct pf_params {
    int version;                /* PF_PARAMS_VERSION */
    int precision;              /* PF_FP64, PF_FP32 or PF_FP32_COMP */
    double dx, eps, tau, dt;    /* dt <= 0: 0.5 x min(tau dx^2/(12 gamma_max T_max), dx^2/(6 D_max)) */
    double gamma2[6];           /* pairs 01 02 03 12 13 23 */
    double gamma3[4];           /* triples 012 013 023 123 */
    double A[4], cE[4][2], kT[4][2], s[4], D[4], TE;
    double T0, G, v;            /* frozen temperature T = T0 + G (z - v t) */
    int seed_layers, n_grains;  /* Voronoi nuclei in the bottom seed_layers planes */
    double window_trigger_z;    /* > 0: shift the window when the interface height reaches it */
    /* general parabolic thermodynamics (version 2) */
    double Am[4][3];            /* A_a as a symmetric positive-definite matrix (a11, a12, a22);
                                   Am[a][0] <= 0: A[a] times the identity */
    double tau_ab[6];           /* relaxation time per phase pair (01 02 03 12 13 23): all > 0, or
                                   all <= 0 for tau everywhere; dt's phi limit takes the smallest */
} pf_params;

typedef struct pf_sim pf_sim;
typedef struct pf_server pf_server;

/* Human-readable text for a status code (static storage).  The paper has no counterpart: status codes
 * are the library's error convention. */
const char *pf_strerror(int status);

/* Parameters of the model of Section 2 (Eq. 1-4) with the fitted parabolic Gibbs energies of Section 3.3;
 * the paper prints no coefficient values (it takes them from its Al-Ag-Cu reference system), so the
 * defaults are a symmetric stand-in.
 * Fill *p with the symmetric parameter set: dx = 1, eps = 4, tau = 1, dt = 0 (auto),
 * gamma2 = 1, gamma3 = 15, A = 1, cE = alpha(0.8,0.1) beta(0.1,0.8) gamma(0.1,0.1)
 * liquid(1/3,1/3), kT = 0 solids / (0.1,0.1) liquid, s = 1 solids / 0 liquid,
 * D = 0 solids / 1 liquid, TE = 1, G = 1e-3, v = 1e-2, T0 = TE - 8 G - 0.15, seed_layers = 8,
 * n_grains = 12, window off, precision PF_FP64.  Returns PF_E_INVAL for p == NULL. */
int pf_default_params(pf_params *p);

/* The paper has no counterpart (allocation of the fields is the library's own concern).
 * Optional allocator hooks for every device buffer the library allocates (fields and
 * scratch).  alloc(bytes, stream, ctx) returns a device pointer or NULL; free(ptr, bytes,
 * stream, ctx) releases it.  Passing NULLs restores cudaMalloc/cudaFree.  Set before
 * pf_create; buffers are released with the hook that allocated them. */
typedef void *(*pf_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*pf_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
int pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void *ctx);

/* The domain of Section 2, discretised into equidistant regular cells, with the two lattices per
 * variable of Section 2.1 (source and destination fields, swapped after each step, Algorithm 1).
 * Create a simulation of nx*ny*nz cells on the current CUDA device.  Allocates the
 * double-buffered phi and mu fields (phi: 4 words/cell, mu: 2 words/cell, words of the
 * chosen precision; twice that for PF_FP32_COMP) and a small device state.  Copies *p;
 * dt <= 0 is replaced by the default limit.  The fields start as pure liquid, mu = 0,
 * t = 0.  stream: a cudaStream_t (NULL: the library creates its own).
 * Errors: PF_E_INVAL (sizes < 1, bad params/version), PF_E_NOMEM, PF_E_CUDA. */
int pf_create(int nx, int ny, int nz, const pf_params *p, void *stream, pf_sim **out);

/* Release every device buffer and handle of sim (waits for its pending work).  No counterpart in the
 * paper: the inverse of pf_create. */
int pf_destroy(pf_sim *sim);

/* The effective parameters, copied into *out, with dt resolved: the explicit Euler scheme of Section 2
 * needs a time step below the stability limits of Eq. 1 and Eq. 3, which the paper does not print. */
int pf_get_params(const pf_sim *sim, pf_params *out);

/* Initial condition (paper Section 2.1, simulation setting): cells with k < seed_layers
 * take the phase of the nearest of n_grains Voronoi seeds drawn from splitmix64(seed)
 * (periodic distance in x and y); liquid above; mu = 0; t = 0; window offset 0. */
int pf_init(pf_sim *sim, uint64_t seed);

/* Advance nsteps explicit steps (Algorithm 1), asynchronously on the sim's stream.
 * Each step: phi-sweep, mu-sweep, FP64 reductions, t += dt, moving-window check.
 * Returns PF_E_INVAL for nsteps < 0, a latched error if one is pending, PF_E_CUDA if a
 * launch fails. */
int pf_step(pf_sim *sim, int nsteps);

/* Wait for the sim's stream; returns and clears the latched error (PF_E_UNSTABLE when a
 * non-finite value appeared in any completed step).  No counterpart in the paper (its kernels run
 * synchronously on the CPU): the library's steps run asynchronously on the device, and this is
 * where their errors surface. */
int pf_sync(pf_sim *sim);

/* The simulation state of Section 3.2: four phi values and two mu values per cell (phi on the Gibbs
 * simplex, Section 2; mu of Eq. 3).
 * Copy the current fields to host FP64 SoA buffers (phi: 4*nx*ny*nz, mu: 2*nx*ny*nz
 * doubles; either may be NULL).  cap_cells must be >= nx*ny*nz.  Synchronising. */
int pf_read_fields(pf_sim *sim, double *phi, double *mu, size_t cap_cells);

/* Overwrite the current fields from host FP64 SoA buffers (both required); time and
 * window offset are left unchanged.  Synchronising. */
int pf_write_fields(pf_sim *sim, const double *phi, const double *mu);

/* As pf_read_fields / pf_write_fields with FP32 host buffers (the single precision the paper uses for
 * the state on disk, Section 3.2) (same SoA layout, half the bytes to
 * move): exact for an FP32 simulation; an FP64 or compensated state is rounded once to FP32 on
 * read (the compensated pair's value), and written values are exact in every precision (the
 * compensated low words become 0).  Errors as the FP64 forms.  Synchronising. */
int pf_read_fields_f32(pf_sim *sim, float *phi, float *mu, size_t cap_cells);
int pf_write_fields_f32(pf_sim *sim, const float *phi, const float *mu);

/* Checkpoint (the paper's infrequent field checkpoints, Section 3.2): write the current fields,
 * simulation time and window offset to the file at path.  Layout: a 64-byte header (magic
 * "PFCKPT01"; int32 version 1, nx, ny, nz, bytes per value, writer precision, planes shifted since
 * init, PF_VARIANT_AUTO's choice of the writer's run (0 none yet, 1 the lean path, 2 the two sweeps);
 * FP64 time and window offset; 8 bytes of padding; little-endian), then for each logical
 * plane k = 0 .. nz-1 the six nx*ny arrays (x fastest) phi_0, phi_1, phi_2, phi_3, mu_0, mu_1.
 * Values are the state's own words, so that nothing is rounded: FP32 for an FP32 simulation, FP64
 * for FP64, and for compensated FP32 (writer precision PF_FP32_COMP, 4 bytes per value) the six
 * arrays of high words followed by the six arrays of low words in each plane (a pair's value is
 * high + low; pairs whose low word lies far below the high word's last bit are not one FP64 value).
 * PF_E_INVAL if the file cannot be written.  Synchronising. */
int pf_checkpoint_write(pf_sim *sim, const char *path);

/* The paper's single-precision checkpoint (Section 3.2: the computation in double precision, the
 * checkpoints in single): the file of pf_checkpoint_write with 4 bytes per value and writer
 * precision PF_FP32, each value of an FP64 or compensated state rounded once to FP32 (an FP32 state
 * is written exactly).  Half the bytes of an FP64 checkpoint; a run resumed from it starts from
 * the rounded state, so it departs from the uninterrupted run by the FP32 rounding (relative
 * 2^-24 of each value) carried forward by the dynamics.  Errors as pf_checkpoint_write. */
int pf_checkpoint_write_f32(pf_sim *sim, const char *path);

/* Restore a checkpoint written for the same grid (any precision: values are converted to this
 * simulation's): fields, time, window offset and shift count; the plane table is rebuilt and no
 * window shift is pending.  A run resumed from a checkpoint of its own precision continues bitwise
 * as the uninterrupted run.  PF_E_INVAL for a missing, short or foreign file or another grid
 * (the fields may then be partly overwritten).  Synchronising. */
int pf_checkpoint_read(pf_sim *sim, const char *path);

/* Phase fractions: phi_a is the fraction of phase a in each cell (Section 2), so its mean over the cells
 * is the phase's volume fraction in the domain (the quantity the Voronoi nuclei of Section 2.1 are drawn
 * for, and the share of each phase in the microstructures of Section 5.2).  The paper prints no
 * reduction; this one accumulates in FP64 on the device so that the sum of many FP32 values keeps its
 * accuracy.  Mean of each phi_a over all cells.  Synchronising. */
int pf_phase_fractions(pf_sim *sim, double out[4]);

/* FP64 diagnostics.  The time t enters the frozen temperature T = T0 + G (z - v t) (Section 3.3); the
 * window offset is the moving window's displacement (Section 3.3); the solute totals are the sums of
 * the concentration c = sum_a h_a c^a(mu, T) whose evolution Eq. 3 states in terms of mu (a closed box
 * keeps them constant); the interface height is the quantity the moving window follows (Section 3.3
 * names the technique but not its trigger: here h_int >= window_trigger_z).  The paper prints no
 * reduction; these accumulate in FP64 on the device.
 * Simulation time t, window offset (planes), solute totals
 * sum_cells c_i with c = sum_a h_a c^a(mu, T), and interface height
 * sum(1 - phi_liquid)/(nx ny).  Any output pointer may be NULL.  Synchronising. */
int pf_stats(pf_sim *sim, double *t, double *window_offset, double solute[2], double *h_int);

/* Planes the moving window (Section 3.3) has moved since pf_init.  Synchronising. */
int pf_window_shifts(pf_sim *sim, int *planes);

/* Interface mesh of one phase (the paper's per-phase isosurface output, Section 3.2): the triangles
 * of the surface phi_phase = iso of the current fields, by marching tetrahedra over the grid of
 * cell centres.  A cube has the centres (i + a, j + b, k + c), a, b, c in {0, 1}, as corners and
 * wraps periodically in x and y (not in z): nx * ny * (nz - 1) cubes, in the order (k ny + j) nx + i.
 * Each cube is cut into the six tetrahedra of its Kuhn triangulation (corner 0, then the axes added
 * in the order of a permutation of (x, y, z), permutations in lexicographic order), so shared faces
 * are cut alike and the surface has no cracks.  A corner is inside when its value is >= iso; a
 * tetrahedron with one inside (or one outside) corner gives one triangle, with two a quad as two
 * triangles; vertices are interpolated linearly along the cut edges; each normal (v1 - v0) x (v2 -
 * v0) points from the inside corners to the outside ones (toward lower phi_phase).  Positions in
 * units of dx, cell (i, j, k) at (i + 1/2, j + 1/2, k + 1/2 + window offset).
 *   phase     0..3 (3 = liquid);  iso  the level, rounded to the simulation's precision (the
 *             compensated FP32 state uses its FP32 words); classification and interpolation run in
 *             that precision, positions are formed in FP64 and stored as FP32
 *   tris      HOST buffer of cap_tris * 9 floats (x, y, z of v0, v1, v2 per triangle), written in the
 *             order cube, tetrahedron, triangle; NULL: count only
 *   ntris     out: the number of triangles (always set on PF_OK and on a too-small buffer)
 * PF_E_INVAL for phase out of range, a non-finite iso, ntris == NULL, or cap_tris below the count
 * (nothing is then written to tris).  Allocates device scratch for the call.  Synchronising. */
int pf_interface_mesh(pf_sim *sim, int phase, double iso, float *tris, size_t cap_tris, size_t *ntris);



/* Kernel classes of the per-kernel timers. */
enum {
    PF_K_PHI = 0,      /* phi-sweep (Eq. 1-2 and the projection) */
    PF_K_MU = 1,       /* mu-sweep (Eq. 3-4) with the FP64 partial sums */
    PF_K_FINALIZE = 2, /* FP64 reduction of the partials, clock, window decision */
    PF_K_POST = 3,     /* plane-table rebuild and fill of planes entering the window */
    PF_K_FUSED = 4,    /* fused phi+mu step (both sweeps in one pass) */
    PF_K_LEAN = 5,     /* the fused step's pure-liquid planes (Section 3.3 shortcuts), a kernel of their own */
    PF_K_PLAN = 6,     /* the fused step's split into pure-liquid and general planes */
    PF_K_GENERAL = 7,  /* the fused step's general planes as the two sweeps (Algorithm 1) */
    PF_K_MESH_COUNT = 8, /* pf_interface_mesh: triangles per segment of cubes */
    PF_K_MESH_SCAN = 9,  /* pf_interface_mesh: offsets of the segments that have triangles */
    PF_K_MESH_EMIT = 10, /* pf_interface_mesh: the triangles */
    PF_K_COUNT = 11
};

/* No counterpart in the paper.  Test hook for the failure path of the bounded device waits: with on != 0 the producer warp of
 * the lean kernel (the fused step's pure-liquid planes) issues none of its copies, so its consumers'
 * waits run out (after about 2^31 clock cycles each), the step ends and pf_sync returns
 * PF_E_TIMEOUT; the fields of the affected planes are then not updated.  The GPU context stays
 * usable; on = 0 restores normal steps.  Not for production use. */
int pf_test_withhold_copies(pf_sim *sim, int on);

/* Kernel variants of pf_step (Algorithm 1's two kernels, or one pass that computes both).  UNFUSED runs
 * Algorithm 1 as two kernels (the phi-sweep writes
 * phi^{n+1}, the mu-sweep reads it back: 88 algorithmic bytes per FP32 cell); FUSED computes
 * phi^{n+1} and mu^{n+1} in one pass (each CTA recomputes phi^{n+1} on a one-cell ring around its
 * tile: 48 bytes per FP32 cell); where the lean kernel can run (FP64, and FP32 with an even nx), FUSED
 * takes the lean path instead: the plan splits each tile's z chunk into pure-liquid planes (the lean
 * kernel, 16 bytes per FP32 cell) and general planes (the two sweeps, run beside the lean kernel).
 * All give the same result up to rounding order (the lean kernel's 7-point form of a pure-liquid cell
 * and the sweeps' flux form round differently).  AUTO (the default) chooses between the lean path and
 * the two sweeps from the state, on the first step after the state was set (pf_init, pf_write_fields*,
 * a checkpoint without a stored choice): with f the fraction of (tile, plane) entries of the current
 * field that are exactly pure liquid, it takes the lean path on domains below 2^20 cells, and when
 * f >= 0.6 (2^20 to 2^23 cells) or f >= 0.45 (larger); where the lean kernel cannot run, the fused tile
 * in FP32 and the two sweeps otherwise.  The choice depends on the state only, so two runs from one
 * state take the same kernels; checkpoints store it, so a resumed run continues as the uninterrupted
 * one.  pf_set_variant(AUTO) makes the choice again at the next step. */
enum { PF_VARIANT_AUTO = 0, PF_VARIANT_UNFUSED = 1, PF_VARIANT_FUSED = 2 };
int pf_set_variant(pf_sim *sim, int variant);

/* Per-kernel device timers (the paper measures kernels separately, Section 5.1).  With
 * enable = 1, every later launch of pf_step is bracketed by CUDA events recorded on the
 * sim's stream; enable = 0 stops recording (pending records are kept).  Not synchronising. */
int pf_profile(pf_sim *sim, int enable);

/* Device milliseconds and launch counts per kernel class (arrays of PF_K_COUNT) accumulated
 * since the last read; resets the accumulators.  Synchronising. */
int pf_profile_read(pf_sim *sim, double ms[], int launches[]);

/* The paper's memory model of a kernel (Section 5.1.1: bytes a cell update must move) applied to
 * these kernels.  Algorithmic HBM bytes per kernel class (array of PF_K_COUNT) of the last step pf_step ran on
 * this simulation (batch steps excluded): the compulsory loads and stores of each kernel.
 *   PF_K_PHI / PF_K_MU (two sweeps): 10 and 12 words a cell (18 and 16 with the compensated low
 *     words), from the cell count;
 *   PF_K_FUSED: 12 words a cell on the planes of the general path, as tallied by the kernel;
 *   PF_K_GENERAL: 22 words a cell on the general planes when they run as the two sweeps beside the
 *     lean kernel (phi^{n+1} goes through HBM there), as tallied by the mu-sweep;
 *   PF_K_LEAN: on the pure-liquid planes (the paper's shortcuts, Section 3.3) 4 words a cell --
 *     mu^n in, mu^{n+1} out; phi^{n+1} = phi^n = e_l is known from the liquid map -- plus 4 words
 *     where phi^{n+1} is stored because the destination buffer does not hold pure liquid there
 *     already; tallied by the kernel (with the fused kernel alone these planes count under
 *     PF_K_FUSED).
 * All zero before the first step.  Synchronising (reads the per-CTA partials back); meant for
 * measurement outside timed regions. */
int pf_step_bytes(pf_sim *sim, double bytes[]);

/*
 * Batched launch.  No counterpart in the paper, whose domain is split into equally sized blocks
 * (Section 3.1) of one simulation; here many independent simulations, each a domain of its own, share
 * every launch.
 * Batched launch: many independent domains of uneven size stepped together.  Each step is one
 * persistent fused kernel whose CTAs pull (domain, tile, z chunk) work items -- largest first --
 * from a device table through an atomic counter, followed by a per-domain FP64 finalize and a
 * per-domain post kernel; steps are replayed from a captured CUDA graph.  Every domain is a
 * pf_sim of its own (fields, clock, window, parameters), reachable with pf_batch_domain for
 * pf_read_fields / pf_write_fields / pf_phase_fractions / pf_stats; it must not be stepped on its
 * own while it belongs to the batch.  All domains share one precision (PF_FP32 or PF_FP64).
 */
typedef struct pf_batch pf_batch;

/* Create ndomains simulations (nx[d] x ny[d] x nz[d] cells, parameters params[d]) on one stream
 * (NULL: the library creates one).  Errors as pf_create; PF_E_INVAL for mixed or compensated
 * precision. */
int pf_batch_create(int ndomains, const int *nx, const int *ny, const int *nz, const pf_params *params,
                    void *stream, pf_batch **out);
int pf_batch_destroy(pf_batch *b);
/* The simulation of domain d (owned by the batch). */
int pf_batch_domain(pf_batch *b, int d, pf_sim **sim);
/* pf_init of every domain with seeds[d]. */
int pf_batch_init(pf_batch *b, const uint64_t *seeds);
/* nsteps steps of every domain (asynchronous).  PF_E_INVAL if a domain was stepped on its own. */
int pf_batch_step(pf_batch *b, int nsteps);
/* Wait for the batch's stream; returns the first latched error of any domain. */
int pf_batch_sync(pf_batch *b);
/* z planes per work item (0: the default, about 6 CTAs of work per SM in total). */
int pf_batch_set_zchunk(pf_batch *b, int zchunk);
/* Autotuner: times trial_steps steps for each candidate launch shape on the batch itself -- z-chunk
 * depth (16 to 512 planes) x persistent general-plane CTAs per SM (1 or 2) x the lean kernel's
 * z-block depth (1, 2 or 4 times the fewest lean CTAs a chunk that keep <= 64 planes a CTA) x its
 * tile (32x8 cells, a liquid-map tile, or 32x4, half of one; the liquid maps, the plan and the
 * general sweeps keep 32x8 tiles) -- (the fields, clocks, windows and plane tables are restored
 * afterwards), keeps the fastest and returns its z-chunk depth in *best (may be NULL) and its measured
 * milliseconds per step in *best_ms (may be NULL); pf_batch_config reports the whole shape. */
int pf_batch_autotune(pf_batch *b, int trial_steps, int *best, double *best_ms);
/* The batch's launch shape: z-chunk depth (0: the default), persistent general-plane CTAs per SM, the
 * lean kernel's split of a z chunk (lean CTAs a chunk / the fewest that keep <= 64 planes a CTA) and
 * the rows of its tile (8 or 4); any pointer may be NULL. */
int pf_batch_config(pf_batch *b, int *zchunk, int *general_ctas_per_sm, int *lean_split, int *lean_tile_rows);
/* Sets the launch shape pf_batch_config reports: zchunk >= 0 (0: each domain's default), general CTAs
 * per SM 1 or 2, lean split 1, 2 or 4, lean tile rows 8 or 4; anything else is PF_E_INVAL.  The shape
 * changes no result: every cell's update is the same arithmetic under any shape. */
int pf_batch_set_config(pf_batch *b, int zchunk, int general_ctas_per_sm, int lean_split, int lean_tile_rows);
/* Algorithmic bytes of the batch's last step, as its kernels tallied them (compulsory traffic of
 * each cell's words, the measure of pf_step_bytes): bytes[0] the general planes' sweeps and the fused
 * tiles, bytes[1] the lean kernel's pure-liquid planes.  Synchronising. */
int pf_batch_step_bytes(pf_batch *b, double bytes[2]);

/*
 * Serving.  No counterpart in the paper: a request loop of the library that runs many independent
 * solidification simulations (each the setting of Section 2.1) on one GPU.
 * Serving: solidification runs submitted as they arrive, run with continuous batching.  A
 * scheduler thread admits queued requests as device memory frees up (admission by HBM footprint
 * of their double-buffered fields against the server's budget; the oldest waiting request keeps
 * a reservation so that large requests are not starved), keeps each run's fields resident, and
 * steps all running requests together with the batched launch in chunks of at most `chunk`
 * steps (a chunk ends where the next request finishes).  Requests arriving meanwhile join at the
 * next chunk boundary.  A request's result does not depend on the mix it ran in: the batched
 * kernel computes each domain exactly as it would alone.  FP32 only.
 */
/* Create a server with a device-memory budget (bytes, 0: 90% of the free memory) and at most
 * max_active concurrently running requests (0: 256); chunk = steps per scheduling round (0: 64).
 * The last two are scheduling knobs of the continuous batching; 0 takes the defaults. */
int pf_server_create(size_t hbm_budget_bytes, int max_active, int chunk, pf_server **out);
/* Stop the scheduler (running requests are cancelled) and release everything. */
int pf_server_destroy(pf_server *srv);
/* Queue a run: nx*ny*nz cells, parameters p (precision must be PF_FP32), Voronoi seed, nsteps
 * steps.  Returns a ticket.  PF_E_NOMEM if the run alone exceeds the budget. */
int pf_submit(pf_server *srv, int nx, int ny, int nz, const pf_params *p, uint64_t seed, int nsteps,
              uint64_t *ticket);
/* Result of a finished run: the phase fractions, the phi slab (4 x nx x ny floats, component
 * major, of the plane z = max(0, floor(h_int) - 8): just inside the solid, where the pattern is
 * frozen; may be NULL), and the latency from submission to completion in seconds (may be NULL).
 * Returns PF_E_PENDING while queued or running, PF_OK once (the record is then released), the
 * run's error (e.g. PF_E_UNSTABLE) if it failed, PF_E_CANCELLED, or PF_E_INVAL for an unknown
 * ticket. */
int pf_poll(pf_server *srv, uint64_t ticket, double fractions[4], float *slab, double *latency_s);
/* Cancel a queued or running request (its record is released on the next pf_poll). */
int pf_cancel(pf_server *srv, uint64_t ticket);
/* Aggregate throughput so far (cell updates / busy seconds / 1e6), running and queued counts and
 * the device bytes held by running requests; any pointer may be NULL. */
int pf_server_stats(pf_server *srv, double *mlups, int *running, int *queued, size_t *used_bytes);

/*
 * Domain decomposition on one device (Section 3.1: the domain is cut into blocks, each with one
 * ghost layer of cells around it; Algorithm 1: after the phi-sweep and after the mu-sweep of every
 * block, the ghost layers take the neighbouring blocks' new boundary layers; Algorithm 2: the
 * exchange of the mu ghost layers runs while the phi-sweep, which does not read them, computes).
 *
 * The domain nx x ny x nz (periodic in x and y) is cut along y into nslabs slabs of
 * floor/ceil(ny / nslabs) rows; slab q owns global rows [floor(q ny / nslabs), floor((q+1) ny / nslabs))
 * and is a pf_sim of nx x (own rows + 2) x nz cells whose first and last rows are ghost rows (the
 * previous and next slab's boundary rows; periodic, so one slab is its own neighbour).  Each step:
 * the phi-sweep of every slab on its own stream; the phi ghost rows copied once both neighbours'
 * phi-sweeps are done; the mu-sweep of every slab once its mu ghost rows have arrived; one kernel
 * that sums the slabs' interface sums, decides the moving-window shift (Section 3.3) for the whole
 * domain and hands it to every slab; each slab's plane table and window fill; the mu ghost rows
 * copied on a separate stream per slab, overlapping the next phi-sweep.  After two steps launched
 * directly, pf_split_step replays the schedule of two steps from a captured CUDA graph.  Every cell is updated by
 * the same arithmetic as in an undivided pf_sim stepped with PF_VARIANT_UNFUSED, so the fields
 * agree with such a run bit for bit (FP32 and FP64).  Ghost-row copies are device-to-device
 * strided copies (cudaMemcpy2DAsync), the stand-in on one GPU for the paper's messages between
 * processes.
 */
typedef struct pf_split pf_split;

/* Create the slabs.  nslabs in [1, ny]; p as for pf_create (dt <= 0: the default for nz).
 * PF_E_INVAL for bad sizes or parameters and for PF_FP32_COMP; PF_E_NOMEM / PF_E_CUDA as pf_create. */
int pf_split_create(int nx, int ny, int nz, const pf_params *p, int nslabs, pf_split **out);
/* Wait for the split's work and release the slabs, streams and events. */
int pf_split_destroy(pf_split *d);
/* The initial state of pf_init(seed) of the undivided domain, in every slab (ghost rows included). */
int pf_split_init(pf_split *d, uint64_t seed);
/* nsteps steps of the whole domain (asynchronous); returns the first latched error. */
int pf_split_step(pf_split *d, int nsteps);
/* Wait for every slab; returns and clears the first latched error (PF_E_UNSTABLE, PF_E_CUDA, ...). */
int pf_split_sync(pf_split *d);
/* The fields of the whole domain, layout as pf_read_fields (cap_cells >= nx ny nz); waits first. */
int pf_split_read_fields(pf_split *d, double *phi, double *mu, size_t cap_cells);
/* Simulation time, window offset (planes), interface height sum(1 - phi_l)/(nx ny) of the current
 * fields of the whole domain (each slab's FP64 sum over its own rows) and the planes shifted so far;
 * any pointer may be NULL; waits first. */
int pf_split_stats(pf_split *d, double *t, double *window_offset, double *h_int, int *planes_shifted);

/*
 * Allocation-free step.  The paper has no counterpart; this entry point serves callers that
 * cannot allocate device memory: code that must live inside a device-memory budget owned by
 * another allocator (a framework's caching pool or a fixed serving arena, where a private
 * cudaMalloc would take memory the owner has already promised elsewhere), and code that must
 * not pay cudaMalloc/cudaFree's implicit device-wide synchronisation in the middle of its work.
 *
 * One explicit step (phi-sweep, then mu-sweep) on caller-owned device fields, asynchronously on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  The call allocates nothing: it
 * calls no cudaMalloc/cudaFree and no allocating library routine.  Its scratch (the step state,
 * the per-plane temperature table and the per-CTA FP64 partial sums) lives in one file-scope
 * device array of PF_NOALLOC_SCRATCH_BYTES, which every GPU that loads this library holds until
 * the process exits.
 *
 *   phi_src, mu_src : the state at time t (device, read only), precision p->precision
 *                     (PF_FP32: float, PF_FP64: double; PF_FP32_COMP is rejected).
 *                     Layout: array of cells in [z][y][x] order, x fastest; a phi cell is 4
 *                     consecutive words (phase 3 = liquid), a mu cell 2 words.  phi buffers
 *                     must be 16-byte aligned, mu buffers 8-byte (FP32) or 16-byte (FP64)
 *                     aligned; misaligned pointers are rejected with PF_E_INVAL.
 *   phi_dst, mu_dst : the state at t + dt (device, written), same layout; must not overlap
 *                     the sources.
 *   t, window_offset: simulation time and window offset (planes) of the source state.  The
 *                     window is never shifted by this call.
 *   h_int_out       : optional host pointer.  When given, the call waits for `stream` and
 *                     stores the interface height sum(1 - phi_l)/(nx ny) of the new state;
 *                     then a non-finite value in the new state returns PF_E_UNSTABLE.
 *
 * Scratch a grid needs, in bytes: 256 (the step state's slot) + 2 nz x 16 w rounded up to a
 * multiple of 256 (the plane table; w = 4 in FP32, 8 in FP64) + 32 x C (one FP64 partial-sum record
 * per CTA of the sweeps), with C = gx gy gz, gx = ceil(nx/32), gy = ceil(ny/8), gz = ceil(nz/zc) and
 * zc = min(nz, max(8, min(64, ceil(nz / ceil(2432 / (gx gy)))))).  Example: 256x256x1024 in FP32
 * needs 256 + 131072 + 32 x 4096 = 262400 bytes, about 0.26 MB.
 *
 * Errors: PF_E_INVAL for null or misaligned fields, sizes < 1, bad parameters, PF_FP32_COMP, or a
 * grid whose scratch exceeds PF_NOALLOC_SCRATCH_BYTES; PF_E_CUDA if a launch fails.
 *
 * Set-up: the first call on each device (with that device current) looks up the scratch
 * array's device address once and keeps it for the life of the process; make that first call
 * before any stream capture.  A caller that resets the device (cudaDeviceReset) invalidates
 * the kept address: do not call this entry point again after a reset in the same process.
 * Every call shares the one array and leaves its contents behind (each call rewrites what it
 * reads before reading it), so calls whose work overlaps on the GPU -- on different streams or
 * different host threads -- race on the scratch and must be serialised by the caller.
 */
#define PF_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
int pf_step_noalloc(int nx, int ny, int nz, const pf_params *p, double t, double window_offset,
                    const void *phi_src, const void *mu_src, void *phi_dst, void *mu_dst, double *h_int_out,
                    void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PF_GB300_H */
