/*
 * hot.h -- C ABI of the GB300 (sm_103a) hashed oct-tree gravity library.
 *
 * The library evaluates the gravitational acceleration and potential of N
 * particles with the treecode of Warren, "2HOT" (SC'13, arXiv:1310.4502):
 *
 *   a_i   =  G sum_{j != i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps^2)^{3/2}
 *   phi_i = -G sum_{j != i} m_j / (|x_j - x_i|^2 + eps^2)^{1/2}
 *
 * (Eq. "eom" with the expansion factor a = 1, Plummer smoothing of Sec.
 * "Force Smoothing"), approximated by Cartesian multipole expansions of order p
 * (Sec. "Multipole Error Bounds", Taylor expansion of the Green's function and
 * moment tensor definition) accepted under an absolute acceleration error bound.
 *
 * Call order, all on the stream given to hot_create:
 *   hot_build_tree      keys, radix sort, hashed oct-tree, sink groups
 *   hot_compute_moments P2M / M2M moments and acceptance-test aggregates
 *   hot_traverse        per-sink-group interaction lists under the tolerance
 *   hot_evaluate_forces M2P + P2P interactions -> acc, pot (original order)
 *   hot_adjoint         dL/dx, dL/dm through the frozen lists (optional)
 * A later call of an earlier stage invalidates the later stages.
 *
 * Pointers: "device" pointers are CUDA device (or managed) memory of the
 * context's device; "host" pointers are ordinary CPU memory.  Arrays are dense
 * and row-major; [N][3] means x0 y0 z0 x1 y1 z1 ...  The library never keeps
 * a caller pointer after a call returns; it owns its tree, moments and lists
 * until the next hot_build_tree or hot_destroy.
 *
 * Errors: every int-returning call returns HOT_OK (0) or a negative HOT_E*
 * code; hot_strerror gives its text.  No call traps the device or aborts the
 * process.  Device-side problems (non-finite input, list scratch overflow,
 * hash-table probe limit, an expired wait) are reported through a status word
 * that the host reads at the synchronisation points named below.
 *
 * Synchronisation: hot_build_tree and hot_traverse synchronise the stream once
 * (they need sizes on the host to allocate); the other calls are asynchronous
 * on the stream unless stated.  The context also owns a second stream: the
 * adjoint's sink pass and, after hot_compute_moments (without background
 * subtraction or order selection), the moment translations and the interaction
 * records run on it beside the work on the caller's stream; every later call
 * except hot_traverse first makes the caller's stream wait for that work, so
 * that a synchronisation of the caller's stream after any call other than
 * hot_compute_moments and hot_traverse covers it (hot_synchronize always does).
 */
#ifndef HOT_H
#define HOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HOT_OK = 0,
    HOT_EINVAL = -1,     /* bad argument (N < 1, p outside [0,8], tol <= 0, eps < 0, ...) */
    HOT_ESTATE = -2,     /* call out of order (e.g. forces before traverse) */
    HOT_ENOMEM = -3,     /* device allocation failed */
    HOT_EOVERFLOW = -4,  /* a capacity limit was still exceeded after the internal retry */
    HOT_ECUDA = -5,      /* a CUDA runtime call failed */
    HOT_EINPUT = -6,     /* non-finite position or mass, or a non-positive total mass */
    HOT_ETIMEOUT = -7    /* a bounded device-side wait gave up */
};

enum { HOT_FP32_MIXED = 0, HOT_FP64 = 1 };

/* Force smoothing (Sec. "Force Smoothing").  A source of mass m at separation d
 * (r = |d|) from a sink gives a = G m f(r^2) d and phi = -G m psi(r):
 *   HOT_SOFT_PLUMMER: f = (r^2 + eps^2)^(-3/2), psi = (r^2 + eps^2)^(-1/2); the
 *     multipole expansions use the same softened kernel.
 *   HOT_SOFT_K1: the K1 compensating kernel of support eps, read as the unit-mass
 *     density 105/(64 pi eps^3) (1 - x^2)(5 - 9 x^2), x = r/eps (zero second moment);
 *     for r < eps, u = r^2/eps^2: f = (175/16 - 147/8 u + 135/16 u^2)/eps^3,
 *     psi = (105 - 175 u + 147 u^2 - 45 u^3)/(32 eps); Newtonian for r >= eps.  The
 *     multipole expansions use the unsoftened kernel and a cell is accepted only
 *     when every source is at least eps from every sink of the group
 *     (|z - g| - Delta_max >= b_max + eps).
 *   HOT_SOFT_SPLINE: the cubic spline kernel of support eps (the kernel of the SPH code
 *     the section cites), the unit-mass density 8/(pi eps^3) w(x), x = r/eps,
 *     w = 1 - 6 x^2 + 6 x^3 (x < 1/2), 2 (1 - x)^3 (1/2 <= x < 1).  For r < eps:
 *     x < 1/2: f = (32/3 - 192/5 x^2 + 32 x^3)/eps^3,
 *              psi = (14/5 - 16/3 x^2 + 48/5 x^4 - 32/5 x^5)/eps;
 *     x >= 1/2, t = 1 - x, M = 1 - 16 t^4 + 128/5 t^5 - 32/3 t^6 (enclosed mass):
 *              f = M/r^3, psi = M/r + (16 t^4 - 64/5 t^5)/eps;
 *     Newtonian for r >= eps; expansions and acceptance as for K1. */
enum { HOT_SOFT_PLUMMER = 0, HOT_SOFT_K1 = 1, HOT_SOFT_SPLINE = 2 };

typedef struct hot_ctx hot_ctx;

typedef struct {
    int p;          /* expansion order, 0..8 (potential terms |a| <= p)           */
    double tol;     /* absolute acceleration error bound per accepted cell, > 0  */
    double eps;     /* softening length, >= 0 (Plummer length, K1 or spline support) */
    double G;       /* gravitational constant                                     */
    int leaf_max;   /* a cell with more particles is refined (levels < 21), >= 1  */
    int group_max;  /* sink groups: topmost cells with <= group_max particles     */
    int precision;  /* HOT_FP32_MIXED or HOT_FP64 interaction arithmetic          */
    int softening;  /* HOT_SOFT_PLUMMER, HOT_SOFT_K1 or HOT_SOFT_SPLINE           */
    int p_min;      /* -1: every accepted cell at order p; 0..p: per-interaction  */
                    /* order selection, the lowest order in [p_min, p] whose      */
                    /* bound E_q(d) <= tol (B_{q+1}, B_{q+2}) accepts the cell     */
    double box;     /* 0: open boundaries; > 0: periodic cube of this side holding */
                    /* every particle (Sec. "Boundary Conditions"): the tree      */
                    /* serves the cube and its images within ws, a local          */
                    /* expansion of order 8 (lattice sums) every farther image;   */
                    /* neutralising background, conducting boundary.  Excludes    */
                    /* p_min >= 0 and the adjoint                                 */
    int ws;         /* periodic: neighbouring cubes on every side served by the   */
                    /* tree, 1..2 (2: the central cube and its 124 neighbours)    */
    double box_lo[3]; /* periodic: lower corner of the cube; every position in   */
                    /* [box_lo, box_lo + box) (not checked: a particle outside    */
                    /* gives forces of no defined meaning, never a fault)         */
    int background; /* 1: background subtraction (Sec. "Background Subtraction"):  */
                    /* the field of the particles minus a uniform density M/L^3  */
                    /* over the tree's root cube (the key frame), see           */
                    /* hot_evaluate_forces; 0: off.  Plummer smoothing, open    */
                    /* boundaries, a fixed order p <= 6 and no adjoint           */
    int bg_up;      /* background subtraction: the surrounding cube of a group is */
                    /* its cell's ancestor bg_up levels up (the root if fewer),   */
                    /* 0..21                                                      */
} hot_params;

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL =
 * legacy default stream).  *out receives the context.  Host-side only; the
 * first call on a device also loads the kernels. */
int hot_create(hot_ctx **out, const hot_params *prm, void *cuda_stream);

/* Replace the parameters (validated as in hot_create).  Changing p, tol, eps,
 * G, precision or softening keeps the tree; changing leaf_max or group_max
 * requires a new hot_build_tree. */
int hot_set_params(hot_ctx *ctx, const hot_params *prm);

/* Morton keys, stable radix sort and hashed oct-tree of N particles
 * (Sec. "Domain Decomposition": space-filling-curve keys turned into a sort;
 * Sec. "Tree Construction and Traversal": cells addressed by key).
 *   pos  device, [N][3] float64, not modified
 *   mass device, [N] float64, not modified
 * Key frame: lo = per-axis minimum, L = largest extent; integer coordinates
 * floor((x - lo) * 2^21 / L) clamped to 2^21 - 1; key = 2^63 | 63 interleaved
 * bits (x highest in each triplet).  Cells are key prefixes; a cell with more
 * than leaf_max particles below level 21 is refined into its non-empty
 * octants.  Cells are stored in depth-first pre-order (children in ascending
 * octant) and inserted into an open-addressed hash table keyed by the cell key
 * (leading placeholder bit: the root key is 1).  Sink groups are the topmost
 * cells that are leaves or hold at most group_max particles.
 * Synchronises the stream once.  Returns HOT_EINPUT for non-finite input. */
int hot_build_tree(hot_ctx *ctx, const double *pos, const double *mass, int64_t N);

/* Moments of every cell about its centre of mass (Eq. "moment tensor":
 * M_a = sum m (x - z)^a, |a| <= p): P2M at the leaves, exact binomial
 * translation (M2M) upwards, in float64; plus the acceptance-test aggregates
 * b_max = max |x - z|, B_{p+1}, B_{p+2} (B_n = sum m |x - z|^n), and the
 * interaction coefficient records.  Under per-interaction order selection
 * (p_min >= 0) also B_n for every n <= p+2 and the records of the orders p_min..p-1.
 * Under background subtraction also every cell's moments about its cube's centre to
 * order p + 2, less those of the uniform cube of density rho = M / L^3 (the contrast),
 * with Q_n = (sum_{|a|=n} n!/a! M_a^2)^(1/2) for n = p+1, p+2 and the contrast's
 * order-p record, and the same for the empty octants of the inner cells (child cubes
 * holding no particle: contrast -rho); this synchronises once (the number of empty
 * octants sizes the records).
 * p in [0, 8], p >= p_min; asynchronous otherwise. */
int hot_compute_moments(hot_ctx *ctx, int p);

/* Group-wise traversal (Sec. "Improving instruction-level parallelism": m
 * source cells x n sink particles) under the absolute-error acceptance test
 * (Sec. "Multipole Error Bounds", geometry of Fig. "mac"):
 *   d = |z_c - g| - Delta_max   (g: centre of the group's bounding box,
 *                                Delta_max: largest distance of a sink from g)
 *   accept cell c for group g  iff  d > b_max and
 *   E(d) = G/d^2 (1 - b_max/d)^-2 [(p+2) B_{p+1}/d^{p+1} - (p+1) B_{p+2}/d^{p+2}] <= tol
 *   (with K1 smoothing also d >= b_max + eps).
 * Under per-interaction order selection a cell is accepted if the bound E_q of some
 * order q in [p_min, p] (B_{q+1}, B_{q+2} in place of B_{p+1}, B_{p+2}) meets tol,
 * and is evaluated at the lowest such order; the order is kept with the list entry.
 * Rejected leaves go to the particle-particle list, rejected inner cells are
 * opened.  Under periodic boundaries every group also traverses the images of the
 * tree within ws cubes (the tree moved by nL, |n|_inf <= ws; in the central one the
 * group's ancestors are opened as above, in the others every cell is tested), each
 * list entry tagged with its image.
 * Under background subtraction a group's surrounding cube S is its cell's ancestor
 * bg_up levels up.  Cells inside S are tested as above; a cell outside S is tested by
 * its contrast about the cube's centre c, d = |c - g| - Delta_max, b = the cube's
 * half-diagonal: accepted iff d > b and
 *   E(d) = G (1 - b/d)^-2 [(p+2) Q_{p+1} / d^{p+3} + (p+3) Q_{p+2} / d^{p+4}] <= tol
 * (an estimate: the bound above needs a positive distribution); a rejected leaf goes
 * to the particle-particle list and its cube to the analytic-cube list, a rejected inner
 * cell is opened; every opened cell outside S (ancestors above S included) adds each
 * empty octant, by its contrast expansion if accepted, else to the analytic-cube list.
 * tol > 0.  Synchronises the stream once (list sizes); HOT_EINVAL under periodic
 * boundaries with 2^24 cells or more. */
int hot_traverse(hot_ctx *ctx, double tol);

/* Interactions on the lists: M2P (expansion of the Plummer-softened kernel, or of
 * 1/r under K1 smoothing; at each entry's order under order selection) and
 * softened P2P (Plummer or K1); sums are kept per sink in float32 with
 * compensated (Kahan) accumulation in the mixed mode, float64 otherwise.  Under
 * periodic boundaries the sources of an image entry are moved by its nL, no sink
 * meets itself outside the central cube, and the far images' local expansion of
 * order 8 (moments of all particles about the cube's centre, the lattice sums of
 * hot_lattice_sums, float32 in the mixed mode) is added.  Under background subtraction
 * the result is the field of the particles less that of the uniform density rho over
 * the root cube [lo, lo + L)^3 (the key frame), the background unsoftened:
 *   a_i = (the softened sum above) - G rho int_root (x - x_i) / |x - x_i|^3 dV,
 *   phi_i = (the softened sum above) + G rho int_root dV / |x - x_i|;
 * each group's analytic cubes and its surrounding cube add the closed-form field of a
 * uniform cube of density -rho at every sink (float32 on float64 corner offsets in the
 * mixed mode).
 *   acc device, [N][3] float64, written in the caller's original order
 *   pot device, [N] float64 or NULL                                      */
int hot_evaluate_forces(hot_ctx *ctx, double *acc, double *pot);

/* Adjoint of L = sum_i g_acc_i . a_i + sum_i g_pot_i phi_i through the frozen
 * lists and frozen expansion centres (moments stay functions of positions and
 * masses).  g_acc device [N][3]; g_pot device [N] or NULL; outputs g_pos
 * device [N][3], g_mass device [N], original order.  Requires a preceding
 * hot_traverse on the same tree.  Orders p <= 6 and a fixed order (HOT_EINVAL
 * for p > 6 or under per-interaction order selection: the coefficient adjoints
 * of one interaction are summed in registers, for one order). */
int hot_adjoint(hot_ctx *ctx, const double *g_acc, const double *g_pot, double *g_pos,
                double *g_mass);

/* Device time in ms of the last call of each stage, measured with CUDA events
 * on the context stream: ms[0] keys+sort, ms[1] tree build, ms[2] moments,
 * ms[3] traversal, ms[4] interactions, ms[5] adjoint.  Synchronises. */
int hot_stage_times(hot_ctx *ctx, float ms[6]);

/* Sizes after the latest stages: out[0] N, [1] cells, [2] sink groups, [3]
 * leaves, [4] deepest level, [5] M2P list entries, [6] P2P list entries
 * (leaves), [7] P2P particle pairs, [8] M2P interactions (entries x sinks),
 * [9] kernels launched by the library since it was loaded (all contexts). */
int hot_sizes(hot_ctx *ctx, int64_t out[10]);

/* Copy an internal array to host memory (for tests).  bytes must equal the
 * array size: see HOT_DBG_* for element type and length.  Synchronises. */
enum {
    HOT_DBG_FRAME = 0,        /* float64[4]: lo_x lo_y lo_z L                */
    HOT_DBG_SORTED_KEYS = 1,  /* uint64[N]: keys in sorted order             */
    HOT_DBG_PERM = 2,         /* int32[N]: original index of sorted slot     */
    HOT_DBG_CELL_KEY = 3,     /* uint64[ncell]                               */
    HOT_DBG_CELL_LEVEL = 4,   /* int32[ncell]                                */
    HOT_DBG_CELL_BEGIN = 5,   /* int32[ncell]: first sorted slot             */
    HOT_DBG_CELL_COUNT = 6,   /* int32[ncell]                                */
    HOT_DBG_CELL_PARENT = 7,  /* int32[ncell] (-1 for the root)              */
    HOT_DBG_CELL_NCHILD = 8,  /* int32[ncell]                                */
    HOT_DBG_GROUP_CELL = 9,   /* int32[ngroup]                               */
    HOT_DBG_GROUP_CENTRE = 10, /* float64[ngroup][3]                         */
    HOT_DBG_GROUP_DMAX = 11,  /* float64[ngroup]                             */
    HOT_DBG_CELL_MASS = 12,   /* float64[ncell]                              */
    HOT_DBG_CELL_COM = 13,    /* float64[ncell][3]                           */
    HOT_DBG_MOMENTS = 14,     /* float64[ncell][ncomp(p)], a by degree, then
                                 a_x descending, then a_y descending         */
    HOT_DBG_CELL_BMAX = 15,   /* float64[ncell]                              */
    HOT_DBG_CELL_B1 = 16,     /* float64[ncell]: B_{p+1}                     */
    HOT_DBG_CELL_B2 = 17,     /* float64[ncell]: B_{p+2}                     */
    HOT_DBG_M2P_OFFSETS = 18, /* int64[ngroup + 1]                           */
    HOT_DBG_M2P_CELLS = 19,   /* int32[n_m2p]                                */
    HOT_DBG_P2P_OFFSETS = 20, /* int64[ngroup + 1]                           */
    HOT_DBG_P2P_CELLS = 21,   /* int32[n_p2p]                                */
    HOT_DBG_M2P_ORDERS = 22,  /* int32[n_m2p]: expansion order of each M2P entry */
    HOT_DBG_M2P_IMAGES = 23,  /* int32[n_m2p]: periodic image of each M2P entry  */
    HOT_DBG_P2P_IMAGES = 24,  /* int32[n_p2p]: periodic image of each P2P entry  */
    /* background subtraction: M2P entries c < ncell are matter expansions, ncell + c the
     * contrast expansion of cell c, 2 ncell + e that of empty octant e; cube entries c <
     * ncell are cell c's cube, ncell + e empty octant e's */
    HOT_DBG_BG_CUBE_OFFSETS = 25, /* int64[ngroup + 1]: the groups' analytic-cube lists */
    HOT_DBG_BG_CUBES = 26,        /* int32[n_cube]                                     */
    HOT_DBG_BG_GROUP_S = 27,      /* int32[ngroup]: the surrounding cube's cell          */
    HOT_DBG_BG_EMPTY_PARENT = 28, /* int32[n_empty]: the cell an empty octant belongs to */
    HOT_DBG_BG_EMPTY_OCTANT = 29  /* int32[n_empty]: its octant (0..7, x highest bit)    */
};
int hot_debug_get(hot_ctx *ctx, int what, void *host_dst, size_t bytes);

/* Sizes of background subtraction after the latest stages: out[0] empty octants, [1]
 * analytic-cube list entries, [2] analytic-cube evaluations (entries x sinks, plus each
 * group's surrounding cube x its sinks), [3] contrast M2P interactions of cells, [4] of
 * empty octants, [5] matter M2P interactions.  HOT_EINVAL when background subtraction is
 * off. */
int hot_bg_sizes(hot_ctx *ctx, int64_t out[6]);

/* Hash-table lookup of n cell keys (host arrays): idx[i] = cell index of
 * keys[i] or -1 when no such cell exists.  Synchronises. */
int hot_lookup(hot_ctx *ctx, const uint64_t *keys, int64_t n, int32_t *idx);

/* Key frame without any allocation.  Computes what hot_build_tree uses as its key
 * frame -- frame[0..2] = per-axis minimum of the positions, frame[3] = L, their
 * largest extent (1 when all coincide) -- and rejects non-finite positions and
 * non-positive masses.  The paper has no counterpart; this entry point exists for
 * callers that must not allocate device memory: hosts that hand out all device
 * memory up front (embedded or real-time loops, memory pools owned by another
 * framework) and must never see cudaMalloc, or code running where the allocator is
 * not reentrant (for instance from inside an allocator callback).  It calls no
 * cudaMalloc, cudaFree or allocating library routine: its
 * scratch (one partial record per 16384 particles, the frame record and a status
 * word) is a fixed device array inside the library (about 200 KB, held by every
 * GPU that loads the library until the process exits).
 *   pos   device, [N][3] float64;  mass device, [N] float64  (inputs, unchanged)
 *   frame device, float64[4]                                  (output)
 *   N     1 .. 2^26; larger N returns HOT_EOVERFLOW (the scratch holds at most
 *         4096 partial records)
 *   cuda_stream  a cudaStream_t (NULL = legacy default stream); the call
 *         synchronises it and copies the input check to host memory before it
 *         returns.
 * The first call on a device looks up the scratch array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one scratch array and it keeps the last call's
 * contents (the status word is cleared at the start of every call): calls that
 * overlap on the GPU -- on different streams, or from different host threads --
 * race and must be serialised by the caller.  Returns HOT_OK, HOT_EINVAL,
 * HOT_EOVERFLOW, HOT_EINPUT or HOT_ECUDA. */
int hot_key_frame_noalloc(const double *pos, const double *mass, int64_t N, double *frame,
                          void *cuda_stream);

/* Synchronise the context stream and return the device status of the calls made since
 * the last synchronisation point: HOT_OK, or HOT_EINPUT, HOT_EOVERFLOW, HOT_ETIMEOUT
 * (a bounded wait of the interaction kernels expired; the kernel skipped the rest of that
 * group's work and the context stays usable), HOT_ECUDA.  The status word is cleared.
 * hot_evaluate_forces and hot_adjoint are asynchronous: their status is reported here or
 * at the next hot_build_tree / hot_traverse. */
int hot_synchronize(hot_ctx *ctx);

/* Test knobs (no counterpart in the paper): they force the library's overflow and
 * timeout paths on small inputs.  Values persist on the context until changed.
 *   HOT_DBGSET_FRONTIER_CAP  per-warp traversal frontier capacity in cells (>= 1); an
 *                            overflow makes hot_traverse retry with 4x the capacity, at
 *                            most three times, then return HOT_EOVERFLOW
 *   HOT_DBGSET_SLOT_CAP      capacity (entries, >= 1) of each group's list slots in the
 *                            one-pass traversal; a group that does not fit makes that call
 *                            fall back to the count/scan/fill passes (the next call sizes
 *                            the slots from the counts)
 *   HOT_DBGSET_WAIT_POLLS    poll limit of the interaction kernels' wait for each staged
 *                            chunk (>= 1; 0 restores the default of 2^22): on expiry the
 *                            warp flags HOT_ETIMEOUT, waits (with the default limit) for
 *                            its copies in flight and leaves its group
 *   HOT_DBGSET_WAIT_PROBE    1: before its first copy, every group's M2P pass waits on a
 *                            barrier that nothing completes (at most min(poll limit, 4096)
 *                            polls), so the wait runs out, HOT_ETIMEOUT is flagged and the
 *                            group is left with no copy in flight; 0: off (default)
 * Returns HOT_OK or HOT_EINVAL. */
enum { HOT_DBGSET_FRONTIER_CAP = 0, HOT_DBGSET_SLOT_CAP = 1, HOT_DBGSET_WAIT_POLLS = 2, HOT_DBGSET_WAIT_PROBE = 3 };
int hot_debug_set(hot_ctx *ctx, int what, int64_t value);

/* y[k] += alpha * x[k] for k < n (device float64 arrays, asynchronous on the
 * context stream).  The kick (v += dt/2 a) and drift (x += dt v) of the
 * kick-drift-kick leapfrog of Sec. "Time Integration", and their adjoints, are
 * this update.  x and y may not overlap unless equal. */
int hot_axpy(hot_ctx *ctx, double *y, const double *x, double alpha, int64_t n);

/* Device memory held by the library's own buffers (tree, moments, records, lists,
 * scratch) over all contexts: out[0] bytes held now, out[1] the largest value since
 * the library was loaded or the peak was last reset; reset_peak != 0 then sets the
 * peak to the current value.  Host-side bookkeeping only (no device call).  The
 * paper has no counterpart: it serves the memory report of multi-step runs. */
int hot_memory_stats(int64_t out[2], int reset_peak);

/* Lattice sums of periodic boundaries (Sec. "Boundary Conditions"): D^g psi_far(0) for
 * every multi-index |g| <= order, psi_far the periodic Green's function of a cube of side
 * L (Ewald conventions: neutralising background, conducting boundary) less the images
 * within ws cubes, 1/|r + nL| for |n|_inf <= ws.  These are the coefficients of the far
 * images' local expansion, computed on the host (no device call).
 *   out  host, far_nc(order) = (order+1)(order+2)(order+3)/6 doubles, graded order: by
 *        |g|, then by descending g_x, then by descending g_y (index n(n+1)(n+2)/6 +
 *        j(j+1)/2 + g_z, n = |g|, j = g_y + g_z)
 * L > 0 finite, ws in 1..2, order in 0..17.  Returns HOT_OK or HOT_EINVAL. */
int hot_lattice_sums(double L, int ws, int order, double *out);

/* Fused-multiply-add throughput microbenchmark (for roofline denominators):
 * runs a register-resident FMA loop on every SM and writes the achieved
 * FLOP/s (FMA = 2) to *flops.  dbl: 0 = float32, 1 = float64.  Synchronises. */
int hot_fma_peak(hot_ctx *ctx, int dbl, double *flops);

/* Text of a HOT_* code (static storage). */
const char *hot_strerror(int code);

/* Free the context and everything it owns (synchronises its stream). */
void hot_destroy(hot_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HOT_H */
