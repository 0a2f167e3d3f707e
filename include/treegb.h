/*
 * treegb.h -- C ABI of the GB300 TreeCode gravity library (libtreegb.so).
 *
 * The library computes, on one GPU, the gravitational accelerations of N
 * particles by the TreeCode (Barnes-Hut) method and advances them with the
 * kick-drift-kick leapfrog, as stated in Sec. 2 of Kuzmin, Sirotin and
 * Khoperskov, "Efficiency of parallel computations of gravitational forces by
 * TreeCode method in N-body models" (2024):
 *   Eq. 1    dv_i/dt = sum_{j != i} G m_j (r_j - r_i) / (|r_j - r_i|^2 + eps^2)^{3/2}
 *   Eqs. 2-5 v += tau/2 a;  r += tau v;  a = a(r);  v += tau/2 a
 *   Sec. 2   octree down to small cells; a far cell acts through its total mass
 *            at its centre of mass (plus, here, its quadrupole); near cells are
 *            summed exactly; theta decides near/far; theta -> 0 gives Eq. 1.
 *
 * Canonical tree (fixed so that the GPU and an independent reference produce
 * the same keys, nodes and interaction lists bit for bit):
 *   box    lo_d = min x_d, L = 2^k the smallest power of two > max_d(hi_d - lo_d)
 *          (L = 1 if all particles coincide), computed in FP64.
 *   keys   q_d = min(2^21-1, floor(fl(x_d - lo_d) * 2^(21-k))); 63-bit key with
 *          bit 3b+2 = bit b of q_x, 3b+1 = q_y, 3b = q_z.
 *   order  ascending (key, original index): a stable radix sort.
 *   octree node 0 = root; a node is internal iff count > leaf_cap and level < 21;
 *          children are the non-empty octants in octant order; breadth-first
 *          numbering (level by level, ascending key prefix within a level).
 *   groups chunks of Gs consecutive sorted particles, cut between neighbours
 *          i-1, i whose keys share P < max(leaf level(i-1), leaf level(i)) -
 *          group_split octal digits, or whose level-P cell holds more than
 *          128 Gs particles; integer box [min q, max q + 1) per axis.
 *   MAC    a node of level l (side s = 2^(21-l), box [c, c+s)) is far for a group
 *          iff s^2 < fl(theta^2 * d2), d2 = sum_d max(0, c_d - ghi_d, glo_d - c_d - s)^2
 *          (exact integers); rejected leaves are summed particle by particle.
 *   cell   y = r_i - R (R = centre of mass), r_s^2 = |y|^2 + eps^2:
 *          a = -G M y/r_s^3 + G Q y/r_s^5 - 5/2 G (y.Q.y) y/r_s^7,
 *          phi = -G M/r_s - 1/2 G (y.Q.y)/r_s^5,
 *          Q = sum m (3 y y^T - |y|^2 I) about R (monopole mode: Q = 0).
 *   phi    phi_i = -sum_{j != i} G m_j / sqrt(|r_ij|^2 + eps^2) for PP terms.
 *
 * Conventions of every call:
 *   - Array arguments are DEVICE pointers owned by the caller, unless marked
 *     "host".  Positions, velocities and accelerations are structure of arrays
 *     [3][n]: x[0..n) then y[0..n) then z[0..n).  Masses and potentials are [n].
 *     All arrays of one workspace have the workspace's precision (TREE_F32 ->
 *     float, TREE_F64 -> double).
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Work is enqueued
 *     on it and the call returns without waiting, except where a call says it
 *     synchronises.
 *   - Arguments are checked before anything is enqueued; a failed check
 *     returns an error and enqueues nothing.
 *   - Errors found on the device (non-finite coordinates, traversal stack
 *     overflow, node capacity exceeded, a wait that timed out) set bits of a
 *     device status word; read them with tree_get_status after the stream has
 *     run.  No C++ exception crosses this interface.
 *   - A workspace is not thread-safe; use one per host thread or serialise.
 *   - n = 0 is valid and enqueues nothing.
 */
#ifndef TREEGB_H
#define TREEGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TREE_OK = 0,
    TREE_ERR_ARG = 1,       /* invalid argument: null pointer, size or parameter */
    TREE_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    TREE_ERR_ALLOC = 3,     /* device memory allocation failed */
    TREE_ERR_CAPACITY = 4,  /* a size exceeds a fixed capacity (the workspace's n_max; the
                               no-allocation direct sum's target limit) */
    TREE_ERR_STATE = 5,     /* call order violated (e.g. tree_forces before tree_moments) */
    TREE_ERR_DEVICE = 6     /* tree_get_status: the device status word is non-zero */
} tree_status_t;

/* Bits of the device status word (tree_get_status). */
#define TREE_DEV_NONFINITE 0x01 /* a coordinate was NaN or infinite */
#define TREE_DEV_STACK     0x02 /* a walk stack overflowed: forces are incomplete */
#define TREE_DEV_NODES     0x04 /* node capacity reached: deep cells became large leaves
                                   (forces stay correct, the tree is not canonical) */
#define TREE_DEV_TIMEOUT   0x08 /* a bounded device-side wait gave up: the results of that call are
                                   invalid (the kernels after the wait returned without work) */
#define TREE_DEV_LIST      0x10 /* interaction-list capacity exceeded */

typedef enum { TREE_F32 = 0, TREE_F64 = 1 } tree_dtype_t;

/* tree_forces flags */
#define TREE_FLAG_EMIT_LISTS 0x1 /* also store the interaction lists (tree_export_lists) */
#define TREE_FLAG_LISTS_ONLY 0x2 /* with EMIT_LISTS: store the lists, skip the force evaluation (a may be NULL) */

typedef struct {
    double G;            /* gravitational constant (Eq. 1) */
    double eps;          /* Plummer softening length, >= 0 (Eq. 1) */
    double theta;        /* opening parameter, >= 0 (Sec. 2); 0 = direct sum */
    int32_t order;       /* 0 = monopole cells, 2 = quadrupole cells */
    int32_t leaf_cap;    /* maximum particles of an internal-free cell, 1..16 (paper: 1) */
    int32_t group_size;  /* particles per walk group: 16, 32 or 64 */
    int32_t stack_depth; /* walk stack entries per warp, 256..8192, a multiple of 32 */
    int32_t precision;   /* TREE_F32 or TREE_F64.  TREE_F32 forms r^-5 for the quadrupole
                            terms: distances up to 2^25 (3.4e7) in the units of x keep it a
                            normal FP32 number; beyond, the quadrupole correction loses
                            precision gradually (the monopole term does not) */
    int32_t kahan;       /* FP32: 1 = compensated per-particle accumulation */
    int32_t group_split; /* delta: cut a group between neighbours that do not share the cell
                            delta levels above the finer of their leaves, or whose smallest
                            common cell holds more than 128 group_size particles;
                            0 = plain chunks */
    int64_t node_cap;    /* node array capacity; 0 = default from n_max and leaf_cap */
} TreeParams;

typedef struct TreeWorkspace TreeWorkspace;

/* Read back after a synchronising call (tree_get_info). */
typedef struct {
    int64_t n;                  /* particles of the last tree_build */
    int64_t n_nodes;            /* nodes of the last tree */
    int32_t depth;              /* deepest level holding a node */
    int32_t box_k;              /* L = 2^box_k */
    double box_lo[3];           /* root corner */
    int64_t level_offset[23];   /* first node of each level 0..21, [22] = n_nodes */
    int64_t pp_pairs;           /* particle-particle pairs evaluated by the last walk */
    int64_t pc_pairs;           /* particle-cell pairs evaluated by the last walk */
    int64_t max_stack;          /* deepest walk stack seen by the last walk */
    int64_t n_groups;           /* walk groups of the last tree */
    int64_t list_pc;            /* stored PC list entries (TREE_FLAG_EMIT_LISTS) */
    int64_t list_pp;            /* stored PP leaf entries (TREE_FLAG_EMIT_LISTS) */
    int64_t launches;           /* CUDA kernels this workspace has launched so far (this call included) */
    int64_t n_segments;         /* independent systems (tree_set_segments); 1 = a single system */
} TreeInfo;

/* Phases timed by tree_timing_read (indices into its ms[] output). */
#define TREE_PHASE_BOX 0     /* box reduction; in leapfrog_step: kick + drift + box (Eqs. 2-3) */
#define TREE_PHASE_KEYS 1    /* Morton keys + radix histograms */
#define TREE_PHASE_SORT 2    /* eight onesweep passes */
#define TREE_PHASE_OCTREE 3  /* level-by-level octree */
#define TREE_PHASE_GATHER 4  /* positions/masses into key order */
#define TREE_PHASE_MOMENTS 5 /* FP64 moments, bottom-up */
#define TREE_PHASE_WALK 6    /* tree walk + forces (+ fused write-back and Eq. 5 kick) */
#define TREE_PHASE_LISTS 7   /* interaction-list count/scan/emit */
#define TREE_PHASE_DIAG 8    /* diagnostics reductions */
#define TREE_PHASE_DIRECT 9  /* direct summation */
#define TREE_PHASE_ADJOINT 10 /* tree_forces_adjoint */
#define TREE_PHASE_H2D 11    /* leapfrog_step_host: copies of the state to the device */
#define TREE_PHASE_D2H 12    /* leapfrog_step_host: copies back after the walk (x's copy overlaps the step;
                                with mapped host arrays only diag's) */
#define TREE_NPHASES 13

/* Fills *p with the defaults: G = 1, eps = 0.01, theta = 0.7, order = 2,
 * leaf_cap = 16, group_size = 32, stack_depth = 1024, precision = TREE_F32,
 * kahan = 1, group_split = 3, node_cap = 0. */
tree_status_t tree_params_default(TreeParams *p);

/* Allocates a workspace for up to n_max particles on the current device.
 * p (host) is copied.  On success *out owns device memory until
 * tree_workspace_destroy.  Errors: TREE_ERR_ARG (bad parameter, n_max < 0),
 * TREE_ERR_ALLOC. */
tree_status_t tree_workspace_create(int64_t n_max, const TreeParams *p, TreeWorkspace **out);
tree_status_t tree_workspace_destroy(TreeWorkspace *ws);

/* Replaces G, eps, theta, order, group_size, kahan and stack_depth (host p).
 * leaf_cap and precision, which shape the stored tree, must stay unchanged
 * (TREE_ERR_ARG otherwise).  A changed leaf_cap needs a new workspace. */
tree_status_t tree_set_params(TreeWorkspace *ws, const TreeParams *p);
tree_status_t tree_get_params(const TreeWorkspace *ws, TreeParams *p);

/* Ensembles (not in the paper, which treats one system): declares that the
 * n = offsets[nseg] particles form nseg independent systems, system b being
 * the caller's particles [offsets[b], offsets[b+1]) (host int64[nseg + 1],
 * offsets[0] = 0, strictly increasing: no empty system; 2 <= nseg <= 65536).
 * Every later build, force and step call treats each system exactly as if
 * it were alone: its own box, keys, octree (its root is node b of level 0),
 * walk groups and walk; there are no forces between systems.  Sorted
 * positions of system b are [offsets[b], offsets[b+1]).  Calls must then pass
 * n = offsets[nseg] (TREE_ERR_ARG otherwise).  nseg = 0 or 1 returns to a
 * single system of any n.  Synchronises the device; drops any captured step
 * and the stored tree.  Errors: TREE_ERR_ARG, TREE_ERR_CAPACITY (n > n_max),
 * TREE_ERR_ALLOC. */
tree_status_t tree_set_segments(TreeWorkspace *ws, int64_t nseg, const int64_t *offsets);
tree_status_t tree_get_segments(const TreeWorkspace *ws, int64_t *nseg);

/* Steps box, keys, sort, octree of the canonical tree (Sec. 2).
 * x: [3][n] positions of dtype (must equal the workspace precision).  The
 * tree (sorted keys, permutation, nodes) stays in ws.  x must stay unchanged
 * until tree_moments has run. */
tree_status_t tree_build(TreeWorkspace *ws, const void *x, int64_t n, int32_t dtype, void *stream);

/* Gathers positions and masses into key order and computes, bottom-up in FP64,
 * every cell's mass, centre of mass and traceless quadrupole (about the centre
 * of mass); rounded copies feed the FP32 walk.  x, m: the arrays of the last
 * tree_build ([3][n], [n]). */
tree_status_t tree_moments(TreeWorkspace *ws, const void *x, const void *m, void *stream);

/* Tree walk and force evaluation for all particles of the last tree: a [3][n]
 * (overwritten), phi [n] or NULL, both in the caller's particle order.
 * flags: TREE_FLAG_EMIT_LISTS additionally stores each group's PC and PP
 * lists in ws (extra device memory, allocated on first use, synchronises
 * the stream once to size it); with TREE_FLAG_LISTS_ONLY as well it stores
 * the lists and evaluates no forces (a and phi are then ignored and may be
 * NULL) -- what the adjoint needs. */
tree_status_t tree_forces(TreeWorkspace *ws, void *a, void *phi, int32_t flags, void *stream);

/* Vector-Jacobian product of the last tree_forces (not part of the paper:
 * gradients through the method).  The tree structure of the last build --
 * key order, cells, walk groups and the interaction lists, which must have
 * been stored by tree_forces(TREE_FLAG_EMIT_LISTS) -- is held fixed; the
 * cell moments are treated as functions of (x, m), so their cotangents are
 * carried back to the particles.  Given a_bar [3][n] (cotangent of the
 * accelerations) and phi_bar [n] or NULL (of the potentials), ADDS the
 * gradient to x_bar [3][n] and m_bar [n] (either may be NULL), all in the
 * caller's order and the workspace precision.  FP64 accumulation of the
 * cotangents.  Scratch is allocated on the first call (about 56 B per
 * particle + 80 B per node).  Errors: TREE_ERR_STATE without stored lists. */
tree_status_t tree_forces_adjoint(TreeWorkspace *ws, const void *a_bar, const void *phi_bar, void *x_bar,
                                  void *m_bar, void *stream);

/* One reverse step of the leapfrog (Eqs. 2-5) through the tree stored in ws,
 * which must have been built at x_{n+1} with lists (tree_build, tree_moments,
 * tree_forces with TREE_FLAG_EMIT_LISTS).  The forward step is
 *   v' = v_n + tau/2 a_n,  x_{n+1} = x_n + tau v',  a_{n+1} = F(x_{n+1}),
 *   v_{n+1} = v' + tau/2 a_{n+1}.
 * On entry x_bar, v_bar hold the cotangents of x_{n+1}, v_{n+1} and a_bar the
 * cotangent of a_{n+1} from its later use (zero at the last step); phi_bar
 * (or NULL) the cotangent of the potentials at x_{n+1}.  The call computes
 *   a_bar += tau/2 v_bar;  (x_bar, m_bar) += VJP of F at x_{n+1};
 *   v_bar += tau x_bar;  a_bar = tau/2 v_bar,
 * leaving the cotangents of x_n, v_n and a_n (= F(x_n)), and accumulating the
 * mass gradient in m_bar.  All [3][n] / [n] device arrays in the caller's order
 * and the workspace precision.  Not part of the paper. */
tree_status_t leapfrog_adjoint_step(TreeWorkspace *ws, void *x_bar, void *v_bar, void *a_bar, void *m_bar,
                                    const void *phi_bar, double tau, void *stream);

/* Vector-Jacobian product of the potential energy W = 1/2 sum m_i phi_i
 * (out[1] of tree_diagnostics; not part of the paper): given w_bar (device
 * double[1], the cotangent of W), writes phi_bar[i] = w_bar m_i / 2 (the
 * cotangent to pass on to tree_forces_adjoint or leapfrog_adjoint_step) and
 * adds w_bar phi_i / 2 to m_bar[i] (the explicit mass dependence at fixed
 * phi).  m, phi, phi_bar, m_bar: device [n] of the workspace precision;
 * phi_bar or m_bar may be NULL. */
tree_status_t tree_energy_vjp(TreeWorkspace *ws, const void *m, const void *phi, const double *w_bar, int64_t n,
                              void *phi_bar, void *m_bar, void *stream);

/* tree_build + tree_moments + tree_forces on (x, m, n). */
tree_status_t tree_accel(TreeWorkspace *ws, const void *x, const void *m, int64_t n,
                         void *a, void *phi, void *stream);

/* One kick-drift-kick step (Eqs. 2-5) in place: v += tau/2 a; x += tau v;
 * a = tree acceleration at the new x; v += tau/2 a.  a holds a^n on entry and
 * a^{n+1} on return; phi [n] (or NULL) receives the potential at the new x.
 * The first kick and the drift are fused with the box reduction, the last
 * kick with the force write-back. */
tree_status_t leapfrog_step(TreeWorkspace *ws, void *x, void *v, const void *m, void *a,
                            void *phi, double tau, int64_t n, void *stream);

/* leapfrog_step on a state held in HOST memory (for callers whose particles
 * live on the host between steps): x, v, a [3][n], m [n] and phi [n] (or
 * NULL) are host arrays of the workspace precision -- page-locked
 * (cudaHostAlloc / cudaHostRegister) for the copies to be asynchronous.  The
 * workspace keeps device copies (allocated on the first call: 44 B per
 * particle of n_max in FP32, 88 in FP64).  The call copies x, v, m, a to the
 * device, runs the step, and copies x, v, a and phi back; x is final after
 * the drift, so its copy back runs on a second stream under the tree build
 * and walk.  When v, a (and phi) are mapped page-locked memory (cudaHostAlloc,
 * or cudaHostRegister with cudaHostRegisterMapped: cudaHostGetDevicePointer
 * succeeds), the walk writes their new values into them directly as it goes
 * and no copy back of them follows the walk.  diag (host double[8], or NULL)
 * receives tree_diagnostics of the new state.  Asynchronous on stream: the host arrays must not be used until
 * the stream has run (the stream waits for every copy). */
tree_status_t leapfrog_step_host(TreeWorkspace *ws, void *x, void *v, const void *m, void *a, void *phi,
                                 double tau, int64_t n, double *diag, void *stream);

/* FP64 reductions over the caller's arrays (precision of ws):
 * out[0] = E_kin = 1/2 sum m |v|^2, out[1] = W = 1/2 sum m phi,
 * out[2..4] = P = sum m v, out[5..7] = L = sum m x cross v.
 * out: device double[8].  Deterministic (fixed reduction order). */
tree_status_t tree_diagnostics(TreeWorkspace *ws, const void *x, const void *v, const void *m,
                               const void *phi, int64_t n, double *out, void *stream);

/* tree_diagnostics per system of the ensemble: out device double[nseg][8].
 * With a single system it equals tree_diagnostics. */
tree_status_t tree_diagnostics_segments(TreeWorkspace *ws, const void *x, const void *v, const void *m,
                                        const void *phi, int64_t n, double *out, void *stream);

/* CUDA graph of one step: captures leapfrog_step(ws, x, v, m, a, phi, tau,
 * n) -- and, when diag is non-NULL, tree_diagnostics into diag (device
 * double[8]) -- on an internal stream; nothing runs.  Every
 * leapfrog_graph_launch then replays that step with the same pointers and
 * parameters as one graph launch on the caller's stream.  A new capture, a
 * tree_set_params or a tree_set_segments drops the graph.  Synchronises the
 * device.  Errors: as leapfrog_step; TREE_ERR_CUDA if capture fails. */
tree_status_t leapfrog_graph_capture(TreeWorkspace *ws, void *x, void *v, const void *m, void *a, void *phi,
                                     double tau, int64_t n, double *diag);
/* TREE_ERR_STATE if no step has been captured. */
tree_status_t leapfrog_graph_launch(TreeWorkspace *ws, void *stream);

/* Autotuner: times one force evaluation (tree_build + tree_moments +
 * tree_forces, `reps` times after one untimed run) on the caller's x, m
 * ([3][n], [n] of base->precision; with nseg > 1 the ensemble given by
 * offsets as in tree_set_segments) for every leaf_cap in {4, 8, 16},
 * group_size in {16, 32, 64} and stack_depth in {512, 1024}, the other
 * parameters taken from base, each leaf_cap in a temporary workspace of
 * n_max = n.  Leaf capacity and group size change the cells that pass the
 * opening criterion of Sec. 2, so they change the force error: every
 * candidate's accelerations are compared with the FP64 direct sum of Eq. 1
 * (each target against its own system) on a fixed sample of up to 512
 * targets (16 systems x 32 for ensembles), and the median relative error
 * |a - a_direct| / |a_direct| is taken.  *best = the fastest candidate whose
 * walks set no device status bit and whose median error is <= max_err
 * (max_err <= 0: no error bound).  table (host double[*ncand][5], may be
 * NULL): rows (leaf_cap, group_size, stack_depth, ms per evaluation, median
 * error), ms = inf for a rejected candidate, error = inf when its walk set a
 * status bit; *ncand in: rows available, out: candidates tried.
 * Synchronises the device.  Errors: TREE_ERR_DEVICE when no candidate
 * qualifies. */
tree_status_t tree_autotune(const TreeParams *base, int64_t nseg, const int64_t *offsets, const void *x,
                            const void *m, int64_t n, int32_t reps, double max_err, TreeParams *best,
                            double *table, int32_t *ncand, void *stream);

/* Boxes of the last build, one per system: lo host double[nseg][3], k host
 * int32[nseg] (L = 2^k); either may be NULL.  Synchronises the device. */
tree_status_t tree_export_boxes(TreeWorkspace *ws, double *lo, int32_t *k);

/* Direct summation of Eq. 1 on the GPU, j != i, for nt targets (indices into
 * x, device int64[nt], each expected in [0, n)) against all n sources.
 * dtype TREE_F32: FP32 pair terms, compensated FP32 sums per source chunk,
 * chunks combined in FP64; TREE_F64: FP64 throughout.  a_out: device double
 * [3][nt]; phi_out: device double [nt] or NULL.  A target index outside
 * [0, n) reads nothing and gets NaN in its outputs.  Uses and overwrites
 * scratch in ws. */
tree_status_t tree_direct_forces(TreeWorkspace *ws, const void *x, const void *m, int64_t n,
                                 int32_t dtype, const int64_t *targets, int64_t nt,
                                 double *a_out, double *phi_out, void *stream);

/* Per-phase GPU timing.  enable != 0 starts (or restarts) accumulation:
 * every later call records CUDA events on its stream around each phase it
 * runs (a few microseconds of host work per phase, no synchronisation).
 * enable = 0 stops recording.  Host-side only; returns TREE_ERR_ARG on a
 * NULL workspace. */
tree_status_t tree_timing_enable(TreeWorkspace *ws, int32_t enable);

/* Synchronises the device and writes the accumulated GPU time per phase
 * since the last tree_timing_enable: ms (host double[TREE_NPHASES]) in
 * milliseconds, calls (host int64[TREE_NPHASES], may be NULL) the number of
 * timed executions of each phase, launches (host int64, may be NULL) the
 * number of kernels launched inside the timed phases. */
tree_status_t tree_timing_read(TreeWorkspace *ws, double *ms, int64_t *calls, int64_t *launches);

/* Direct summation like tree_direct_forces, for callers that cannot allocate
 * device memory: it needs no workspace and calls no allocator.  This entry
 * has no counterpart in the paper; it exists for applications whose own
 * memory pool owns the GPU, or code that may only touch buffers it is given.
 * x [3][n], m [n] of dtype; targets device int64[nt], each expected in
 * [0, n) (an index outside gets NaN outputs and reads nothing); G, eps as
 * for tree_direct_forces; a_out device double [3][nt]; phi_out device double
 * [nt] or NULL.
 * Scratch is a fixed 4 MiB array inside the library, present on every GPU
 * that loads it until the process exits.  At most TREE_NOALLOC_MAX_TARGETS
 * targets per call (TREE_ERR_CAPACITY beyond); any n >= 1 sources.
 * The first call on each device looks up that array's device address (make
 * it before any stream capture).  All calls share the one array: calls that
 * may overlap on the GPU (different streams, or different host threads)
 * race and give wrong results; serialise them.  Nothing needs clearing
 * between calls: every scratch entry is written before it is read. */
#define TREE_NOALLOC_MAX_TARGETS 4096
tree_status_t tree_direct_forces_noalloc(const void *x, const void *m, int64_t n, int32_t dtype, double G,
                                         double eps, const int64_t *targets, int64_t nt, double *a_out,
                                         double *phi_out, void *stream);

/* Bounded waits (not part of the paper).  Every device-side wait of the build
 * (the decoupled look-backs of the sort passes, the octree levels and the
 * walk-group scan) gives up after a limit of clock cycles: it then sets
 * TREE_DEV_TIMEOUT, the rest of its own kernel writes only in bounds, and
 * every later kernel of that build, force or gradient call returns without
 * touching the tree -- the call's results are invalid, the context stays
 * usable and the next build starts clean.  wait_cycles > 0 sets the limit
 * (default 2e9 cycles, about 1 s); 0 keeps it.  withhold_pass and
 * withhold_tile >= 0 make that tile of that sort pass (0..9) skip publishing
 * its look-back words, so the tiles after it run into the limit: a test of
 * the timeout path that needs no fault; -1 for both turns it off.
 * Synchronises the device.  Errors: TREE_ERR_ARG. */
tree_status_t tree_set_waits(TreeWorkspace *ws, int64_t wait_cycles, int32_t withhold_pass, int64_t withhold_tile);

/* Synchronises the device, returns TREE_OK if the device status word is 0,
 * else TREE_ERR_DEVICE; *status (host) receives the word.  clear != 0 resets
 * it to 0 afterwards. */
tree_status_t tree_get_status(TreeWorkspace *ws, int32_t *status, int32_t clear);

/* Synchronises the device and fills *info (host). */
tree_status_t tree_get_info(TreeWorkspace *ws, TreeInfo *info);

/* Copies the last tree into caller device buffers (any may be NULL):
 * keys: uint64[n] sorted keys; perm: uint32[n], sorted position -> caller
 * index; level: int32[n_nodes]; corner: uint32[3][n_nodes]; first, count:
 * uint32[n_nodes] (range of sorted particles); child: int32[n_nodes] first
 * child or -1; nchild: int32[n_nodes]. */
tree_status_t tree_export_tree(TreeWorkspace *ws, uint64_t *keys, uint32_t *perm, int32_t *level,
                               uint32_t *corner, uint32_t *first, uint32_t *count,
                               int32_t *child, int32_t *nchild, void *stream);

/* Copies the moments of the last tree_moments into caller device buffers
 * (any may be NULL): M [n_nodes], R [3][n_nodes], Q [6][n_nodes] ordered
 * (xx, yy, zz, xy, xz, yz), FP64. */
tree_status_t tree_export_moments(TreeWorkspace *ws, double *M, double *R, double *Q, void *stream);

/* Copies the lists stored by tree_forces(TREE_FLAG_EMIT_LISTS) into caller
 * device buffers: pc_off, pp_off int64[n_groups+1] (CSR offsets), pc_list
 * int32[list_pc] (far cells), pp_list int32[list_pp] (near leaves).  Within a
 * group, entries are in walk order, not sorted. */
tree_status_t tree_export_lists(TreeWorkspace *ws, int64_t *pc_off, int32_t *pc_list,
                                int64_t *pp_off, int32_t *pp_list, void *stream);

/* Copies the lists of selected groups only (what tree_export_lists gives for
 * those groups): gsel (host int64[nsel], each 0 <= gsel[k] < n_groups) names
 * the groups; pc_off, pp_off (host int64[nsel+1]) receive CSR offsets in
 * selection order; pc_list, pp_list (device int32, capacity pc_off[nsel],
 * pp_off[nsel]) receive the far-cell and near-leaf entries of group gsel[k]
 * at [off[k], off[k+1]), in walk order.  With pc_list = pp_list = NULL only
 * the offsets are written (to size the buffers).  Synchronises the stream.
 * Errors: TREE_ERR_STATE without stored lists, TREE_ERR_ARG for a group out
 * of range. */
tree_status_t tree_export_lists_groups(TreeWorkspace *ws, int64_t nsel, const int64_t *gsel, int64_t *pc_off,
                                       int32_t *pc_list, int64_t *pp_off, int32_t *pp_list, void *stream);

/* Copies the per-group records of the last walk into a caller device buffer
 * out (uint32 [4][n_groups]): row 0 far cells (PC list length), row 1 near
 * particles (PP sources, self included), row 2 deepest walk stack, row 3
 * near leaves. */
tree_status_t tree_export_group_stats(TreeWorkspace *ws, uint32_t *out, void *stream);

/* Copies the walk groups of the last tree_build into gfirst (device
 * uint32[n_groups + 1]): group g is sorted particles [gfirst[g], gfirst[g+1]),
 * gfirst[n_groups] = n.  Synchronises to read n_groups. */
tree_status_t tree_export_groups(TreeWorkspace *ws, uint32_t *gfirst, void *stream);

/* Host only, no device work: the integer thresholds D_l (l = 0..21) with
 * "node of level l is far" <=> d2 >= D_l, where D_l = min{d : s_l^2 < fl(theta^2 d)}.
 * D (host int64[22]); theta = 0 gives INT64_MAX everywhere. */
tree_status_t tree_mac_table(double theta, int64_t *D);

/* Measured FP32 FMA throughput of the current GPU in TFLOP/s (2 flops per
 * FMA), the roofline denominator of the FP32 walk (not part of the paper):
 * register-only chains of fmaf (scalar) and of packed __ffma2_rn (packed) in
 * four waves of resident blocks, best of three timed launches after one
 * warm-up.  Either pointer (host) may be NULL.  Synchronous; takes well
 * under a second. */
tree_status_t tree_fp32_peak(double *tflops_scalar, double *tflops_packed);

/* Static string for a status code. */
const char *tree_status_string(tree_status_t s);

/* Library version, e.g. "treegb 0.1". */
const char *tree_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TREEGB_H */
