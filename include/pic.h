/*
 * pic.h -- C ABI of libpic: the particle step of particle-in-tree (PIT) and
 * particle-in-dual-tree (PIDT) on a k = 3 spacetree, for one GB300 (sm_103a).
 *
 * Method: Weinzierl, Verleye, Henri, Roose, "Two Particle-in-Grid Realisations
 * on Spacetrees", arXiv:1508.02435.  One time step is the PIC cycle of
 * Section 3: deposit rho = sum_i R(x_i) with d-linear R (item 1), solve
 * L(V) = rho (item 2, auxiliary: a caller hook or built-in Jacobi sweeps),
 * E = -grad V and gather E_i = R^T(x_i) E (item 3), push d_t v = (q/m) E,
 * d_t x = v (item 4), then re-bin every particle -- with no bound on how many
 * cells it moved -- into the leaf that covers it (PIT, Algorithm 1 / Theorem 1)
 * or into the dual cell of the vertex on that leaf's level that covers it
 * (PIDT, Algorithms 2-3 / Theorem 2).  Buckets are stable: stayers keep their
 * order at the head of their bucket, movers follow in storage order.
 *
 * Conventions shared by every call:
 *   - Domain [0,1)^d, d in {2,3}, periodic.  k = 3: a refined cell has 3^d
 *     children, local digit l = i0 + 3 i1 + 9 i2 (x fastest) (Section 4).
 *   - Arrays of particle or vertex quantities are structure-of-arrays,
 *     [axis][n] (axis-major, each axis contiguous).
 *   - `where` = PIC_HOST (pageable or pinned host memory) or PIC_DEVICE
 *     (device memory of the handle's device).  The library never keeps a
 *     pointer it was given; inputs are copied, outputs are written before the
 *     call returns (host) or are stream-ordered on the handle's stream (device).
 *   - Every call returns PIC_OK (0) or a negative PIC_E* code; no exception or
 *     signal crosses the ABI.  pic_last_error() gives a message per handle
 *     (with NULL: the last failed pic_load of the calling thread).
 *   - Leaves are numbered in depth-first pre-order (children in digit order);
 *     finite-element vertices (non-hanging grid points) by row-major position
 *     on the finest level; PIDT owner vertices by (level, row-major index).
 *   - The library owns all device memory it allocates (at create, re-tree,
 *     re-refinement, autotuning); pic_destroy frees it.  It is taken with
 *     cudaMalloc, or from the caller's allocator set by pic_set_allocator.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PIC_API __attribute__((visibility("default")))
#else
#define PIC_API
#endif

#define PIC_OK 0
#define PIC_EINVAL (-1)    /* malformed argument or tree (refined node without 3^d children,
                              depth > 18, d not 2 or 3, count mismatch) */
#define PIC_ENOMEM (-2)    /* device or host allocation failed */
#define PIC_ERANGE (-3)    /* non-finite position or velocity */
#define PIC_EHOOK (-4)     /* the field-solve hook returned non-zero */
#define PIC_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define PIC_ECUDA (-6)     /* a CUDA runtime call failed */
#define PIC_ESTATE (-7)    /* call not valid in the handle's state */
#define PIC_EIO (-8)       /* checkpoint file missing, unreadable, truncated or corrupt */

#define PIC_PIT 0
#define PIC_PIDT 1
#define PIC_FP64 0        /* positions and arithmetic in FP64 */
#define PIC_FP32_SPLIT 1  /* leaf index + FP32 cell-local offset, FP32 arithmetic */
#define PIC_HOST 0
#define PIC_DEVICE 1

typedef struct pic_s *pic_t;

/* Spacetree as level-order (breadth-first) refinement flags: flags[i] = 1 if
 * node i is refined.  Node 0 is the root; the children of a refined node
 * follow in digit order after all children of earlier refined nodes
 * (Section 4).  flags is host memory. */
typedef struct {
  int32_t d;
  int64_t n_nodes;
  const uint8_t *flags;
} pic_tree_desc;

/* Particles: n positions x[d][n] in [0,1)^d (wrapped on input) and velocities
 * v[d][n], FP64, in host or device memory per `where`. */
typedef struct {
  int64_t n;
  const double *x;
  const double *v;
  int32_t where;
} pic_particles_desc;

typedef struct {
  int32_t scheme;     /* PIC_PIT or PIC_PIDT */
  int32_t precision;  /* PIC_FP64 or PIC_FP32_SPLIT */
  double q;           /* charge per particle */
  double qm;          /* charge / mass */
  double ion;         /* uniform neutralising background density (Appendix A) */
  int32_t sweeps;     /* damped Jacobi sweeps of the built-in solve per step */
  double omega;       /* Jacobi damping factor */
  int32_t track_ids;  /* 1: carry input particle ids through the re-bin (pic_bins) */
  void *stream;       /* cudaStream_t for every kernel of the handle; NULL = default */
  int32_t path;       /* PIC_PATH_AUTO (brick path where it applies) or PIC_PATH_GENERIC */
} pic_config;

#define PIC_PATH_AUTO 0     /* uniform tree + PIT + split precision: two-pass brick kernels */
#define PIC_PATH_GENERIC 1  /* per-particle push + counting-sort re-bin, any tree */

/* Optional field-solve hook, called once per step with the vertex charges
 * Q[n_vertices] (FP64, or FP32 in split mode) and a buffer E[d][n_vertices]
 * to fill with the field at the vertices.  It must only enqueue work on
 * `stream` (no synchronisation) and return 0, else the step fails PIC_EHOOK. */
typedef int (*pic_solve_fn)(void *user, const void *Q_dev, void *E_dev, int64_t n_vertices,
                            int32_t precision, void *stream);

typedef struct {
  int32_t d, scheme, precision, depth;
  int64_t n_particles;
  int64_t n_leaves;
  int64_t n_vertices;    /* finite-element vertices (non-hanging) */
  int64_t n_buckets;     /* leaves (PIT) or PIDT owner vertices */
  int64_t n_keys;        /* sort keys: leaves (PIT) or owner vertex x 2^d quadrants (PIDT) */
  int32_t uniform;       /* 1 if every leaf is on `depth` */
  int32_t brick;         /* 1 if steps run the brick path */
  int32_t n_instances;   /* independent plasmas in the handle (1 unless batched) */
  int64_t device_bytes;  /* device memory held by the handle */
} pic_info_t;

typedef struct {
  int64_t step;          /* steps taken */
  int64_t movers;        /* particles whose key changed in the last step */
  int64_t max_bucket;    /* largest bucket after the last re-bin */
  double total_charge;   /* FP64 sum of the vertex charges of the last deposit */
  double residual;       /* FP64 2-norm of b - A V after the last built-in solve */
  int32_t error;         /* sticky device error: PIC_ERANGE if a non-finite value was seen,
                            PIC_ETIMEOUT if a bounded device wait gave up */
  int64_t tunnellers;    /* with lift counting on (pic_count_lifts): particles whose new leaf
                            does not touch their old leaf (moved two cells or more on the finer
                            level), summed over the counted steps; -1 when counting is off */
} pic_stats_t;

/* Device memory through the caller's allocator, for example PyTorch's caching
 * allocator.  alloc(user, bytes, stream) returns device memory of the current
 * device, aligned to 256 bytes, or NULL (the calling function then fails with
 * PIC_ENOMEM); free_fn(user, ptr, bytes, stream) returns it.  `stream` is the
 * handle's stream: the library synchronises it after each allocation (a
 * recycled block may still be in use by work queued before) and before
 * returning blocks, so a stream-ordered pool may hand a block to the next
 * user on that stream at once.  The setting is process-wide and
 * taken by handles created afterwards, which keep it for all their later
 * allocations and frees; both NULL restores cudaMalloc / cudaFree.  Only one
 * of the two NULL: PIC_EINVAL.  Host only; no device call.  The paper has no
 * counterpart: a library utility. */
typedef void *(*pic_alloc_fn)(void *user, size_t bytes, void *stream);
typedef void (*pic_free_fn)(void *user, void *ptr, size_t bytes, void *stream);
PIC_API int pic_set_allocator(pic_alloc_fn alloc, pic_free_fn free_fn, void *user);

/* Create a handle on the current CUDA device: the problem statement of
 * Section 3 (particles with positions and velocities in a domain covered by
 * a spacetree, Section 4) and of Section 5's introduction (every particle held
 * by the leaf, PIT, or the vertex, PIDT, that covers it).  Validates and
 * tabulates the tree (refined nodes with 3^d children, depth <= 18, d in
 * {2, 3}; else PIC_EINVAL), copies the particles (host or device per
 * parts->where; non-finite values: PIC_ERANGE), and bins them: initial key
 * (Theorem 1 / Theorem 2 end state) and stable bucket sort (every particle
 * counts as moved, so buckets keep input order).  *out receives the handle,
 * NULL on failure.  Memory: PIC_ENOMEM; CUDA failures: PIC_ECUDA. */
PIC_API int pic_create(pic_t *out, const pic_tree_desc *tree, const pic_particles_desc *parts,
               const pic_config *cfg);
/* Free every device buffer of the handle (through the allocator it was
 * created with) after its stream has drained; NULL is ignored.  The paper's
 * grid and particle containers have no counterpart to release: a library
 * utility. */
PIC_API void pic_destroy(pic_t h);
/* Error text of a return code, and the message of the handle's last failure
 * (NULL handle: of the last failed creation on this thread); sizes and mode
 * of a handle.  Library utilities without a counterpart in the paper. */
PIC_API const char *pic_strerror(int code);
PIC_API const char *pic_last_error(pic_t h);
PIC_API int pic_info(pic_t h, pic_info_t *out);

/* Batch of n_inst independent plasmas of uneven size with uniform trees of
 * any depth (same d): trees[i], parts[i], charge per particle q[i] (NULL:
 * cfg->q for all).  No counterpart in the paper (each instance is the problem
 * of pic_create; the batch fills one GPU with many small ones).  Leaves, vertices, buckets and particles are concatenated
 * instance by instance; every phase of a step is one launch over the whole
 * batch.  Particle ids run over the batch in input order. */
PIC_API int pic_create_batch(pic_t *out, int32_t n_inst, const pic_tree_desc *trees,
                             const pic_particles_desc *parts, const double *q, const pic_config *cfg);

/* Per-instance offsets (no counterpart in the paper) into the concatenated
 * particle storage, vertex arrays and bucket list; each array has n_instances + 1 entries (host memory, any
 * may be NULL).  Particle ranges are fixed: no particle leaves its instance. */
PIC_API int pic_instances(pic_t h, int64_t *particle_start, int64_t *vertex_start, int64_t *bucket_start);

/* Leapfrog start: v_{-1/2} = v_0 - (q/m) E(x_0) dt/2 (deposit, solve, gather):
 * the time integration of Section 3 item 4 read as leapfrog. */
PIC_API int pic_init_leapfrog(pic_t h, double dt, pic_solve_fn hook, void *user);

/* One PIC step (Section 3 items 1-4) plus the PIT/PIDT re-bin (Section 5),
 * enqueued on the handle's stream.  Asynchronous; pic_sync reports errors. */
PIC_API int pic_step(pic_t h, double dt, pic_solve_fn hook, void *user);

/* Only the timed hot path of a step, with the field E held fixed from the last
 * solve: deposit of the current positions (Section 3 item 1), gather + push
 * (items 3-4), key and re-bin (Section 5). */
PIC_API int pic_step_fixed_field(pic_t h, double dt);

/* The particle-handling step of the paper's experiments (Section 6): no
 * field solve and no particle-grid interplay -- every particle moves by its
 * own velocity, x <- x + v dt, then is re-binned (PIT / PIDT) like after a
 * PIC push.  boundary = PIC_PERIODIC wraps the unit box; PIC_REFLECT
 * reflects at its walls without any other change of the velocity (the
 * velocity component is negated after an odd number of wall hits; a particle
 * landing exactly on the far wall is placed just inside it).  flops (0 ..
 * 65536) artificial floating-point operations are spent per particle move
 * (the paper's 0-4096 flops per move); they do not change any result.  The
 * brick path is not used for this step (its kernels gather the field); lift
 * counting applies.  Invalid boundary, flops or dt: PIC_EINVAL.  Drops
 * captured graphs.  Asynchronous. */
#define PIC_PERIODIC 0
#define PIC_REFLECT 1
PIC_API int pic_step_particles(pic_t h, double dt, int32_t boundary, int32_t flops);

/* No counterpart in the paper (launch machinery of this library).  Capture
 * the fixed-field step (deposit when due, gather + push + key, re-bin) as
 * CUDA graphs after one ordinary step; the handle's stream must
 * not be the legacy default stream.  Two graphs are kept because a step
 * swaps ping-pong buffers.  Any call that rebuilds buffers (re-tree, tuning)
 * drops them. */
PIC_API int pic_graph_capture(pic_t h, double dt);

/* The same for the whole time step with the built-in solve (no hook): deposit
 * when due, Jacobi sweeps + vertex field, gather + push + key, re-bin.  A
 * replay is one pic_step(h, dt, NULL, NULL), bit for bit. */
PIC_API int pic_graph_capture_step(pic_t h, double dt);

/* Replay `steps` captured steps on the handle's stream (asynchronous). */
PIC_API int pic_graph_launch(pic_t h, int32_t steps);

/* Launch tuning (no counterpart in the paper).  Tuning = {path (1 brick, 0
 * generic), threads per block of the push, of
 * the per-leaf deposit, of the per-vertex kernels}.  pic_autotune times
 * every candidate for `trials` fixed-field steps on the handle's own
 * particles, keeps the fastest and restores the particle state; the chosen
 * values go to tuned[4] (may be NULL).  pic_set_tuning applies stored values
 * (for example from a cache); pic_get_tuning reads the current ones. */
PIC_API int pic_autotune(pic_t h, double dt, int32_t trials, int32_t *tuned);
PIC_API int pic_set_tuning(pic_t h, const int32_t *tuned);
PIC_API int pic_get_tuning(pic_t h, int32_t *tuned);

/* Wait for the handle's stream; returns the sticky device error if any
 * (PIC_ERANGE, PIC_ETIMEOUT when a bounded device wait gave up).  A library
 * utility without a counterpart in the paper. */
PIC_API int pic_sync(pic_t h);

/* Failure detection of device waits (no counterpart in the paper; a library
 * safeguard).  Every device-side wait of the library is bounded: the brick
 * kernels wait for their bulk copies at most `cycles` SM clocks (default 4e9,
 * about two seconds), then record PIC_ETIMEOUT (reported by pic_sync) and
 * return after the copies in flight have landed, leaving the context usable.
 * pic_set_wait_limit sets the limit of the handle's later steps (1e3 <=
 * cycles <= 2^40, else PIC_EINVAL) and drops captured graphs.
 * pic_wait_selftest runs, on `stream`, one CTA whose barrier expects 16 bytes
 * that are never sent and waits for them with the same bounded wait: it
 * returns PIC_ETIMEOUT when the wait gave up and the kernel returned (the
 * expected outcome), PIC_OK if the barrier completed, PIC_ECUDA on a CUDA
 * error.  Synchronous; allocates one 4-byte flag. */
PIC_API int pic_set_wait_limit(pic_t h, int64_t cycles);
PIC_API int pic_wait_selftest(int64_t cycles, void *stream);

/* Vertex charges Q[n_vertices] of the current positions: Section 3 item 1,
 * rho = sum_i R(x_i) with d-linear R on the leaf that covers x_i, as the
 * finite-element load Q_v = q sum_i phi_v(x_i) + ion integral(phi_v) (hanging
 * vertices pass their share to the vertices of the coarse face).  FP64 values
 * in both precisions, summed in a fixed order (no floating-point atomics), so
 * the result is run-to-run identical.  Q_out is caller-owned, host or device
 * per `where`.  Computes the deposit if the positions changed since the last
 * one.  pic_field / pic_potential return E[d][n_vertices] and V[n_vertices]
 * of the last solve (Section 3 items 2-3). */
PIC_API int pic_deposit(pic_t h, double *Q_out, int32_t where);
PIC_API int pic_field(pic_t h, double *E_out, int32_t where);
PIC_API int pic_potential(pic_t h, double *V_out, int32_t where);

/* Buckets after the last re-bin -- the association of particles with leaves
 * (PIT, Section 5.1) or dual cells of vertices (PIDT, Section 5.2), stored as
 * the paper's per-cell particle arrays (Section 4.2) in one CSR layout:
 * bucket_start[n_keys + 1] offsets into the storage order (PIT: one bucket
 * per leaf; PIDT: per owner vertex and quadrant, key = vertex 2^d + quadrant)
 * and perm[n] the input particle id stored at each position (needs
 * track_ids, else PIC_ESTATE when perm is not NULL).  Caller-owned, host or
 * device per `where`. */
PIC_API int pic_bins(pic_t h, int64_t *bucket_start, int32_t *perm, int32_t where);

/* Sort keys per particle in storage order: the PIT leaf (Section 5.1) or the
 * PIDT owner vertex (Section 5.2) as leaf id, or owner vertex * 2^d +
 * quadrant.  Caller-owned, host or device per `where`. */
PIC_API int pic_keys(pic_t h, int32_t *keys, int32_t where);

/* Particles in storage order: absolute FP64 positions x[d][n] in [0, 1)^d
 * (split mode: (c + o) / 3^level from the leaf coordinates c and the cell
 * offset o) and FP64 velocities v[d][n] -- the particle state of Section 3
 * (position and velocity per particle).  Caller-owned, host or device per
 * `where`; either pointer may be NULL. */
PIC_API int pic_get_particles(pic_t h, double *x, double *v, int32_t where);

/* Native state in storage order (the particle state of Section 3 in the
 * handle's precision), for checkpoints and host round trips.
 * FP64: x[d][n], v[d][n] (double).  Split: leaf[n] (int32), o[d][n], v[d][n]
 * (float).  Unused pointers may be NULL.  pic_set_state replaces the particles
 * (same n) and re-bins them. */
PIC_API int pic_get_state(pic_t h, int32_t *leaf, void *x_or_o, void *v, int32_t where);
PIC_API int pic_set_state(pic_t h, const int32_t *leaf, const void *x_or_o, const void *v,
                  int32_t where);

/* Counters of the last step: movers (particles whose key changed -- the
 * PIDT `moved` flag of Section 5.2, for PIT the particles that left their
 * leaf), the largest bucket, the FP64 charge total of the last deposit (the
 * neutrality check of Section 3 item 1 against the ion background of
 * Appendix A), the residual norm of the last built-in solve (item 2), the
 * step count and the sticky device error.  Synchronous. */
PIC_API int pic_stats(pic_t h, pic_stats_t *out);

/* Lift and drop counts (the paper's cost measure for particle handling,
 * Section 6: lifting a particle n levels counts as n lifts).  With counting
 * on, every pic_step / pic_step_fixed_field adds per particle:
 *   PIT (Algorithm 1): for a particle that went from leaf L1 to leaf L2,
 *     lifts = level(L1) - m and drops = level(L2) - m, m the level of the
 *     deepest common ancestor of L1 and L2 (it is lifted out of every cell
 *     that no longer covers it and dropped into every cell that does);
 *   PIDT (Algorithms 2-3, read as a count): none for a particle whose new
 *     owner vertex is a vertex of its old leaf on that leaf's level (handed
 *     over inside the cell); otherwise lifts from the old owner vertex to the
 *     deepest vertex of the dual tree whose dual cell holds both owners' dual
 *     cells (the dual parent of (l, j) is (l - 1, (j + 1) div 3)) and drops
 *     from there to the new owner;
 *   both: a tunneller when L2 does not touch L1 (the closed boxes share no
 *     point, periodic).
 * Stayers add nothing.  Two or three extra kernels per step; handles with
 * track_ids only, PIDT ones with a single instance (PIC_ESTATE otherwise);
 * graph capture is refused while counting.  pic_count_lifts(h, 1) starts (or
 * restarts) from zero, (h, 0) stops and frees the counters.  pic_lift_counts
 * returns the totals and the steps counted since the start (synchronous;
 * PIC_ESTATE when counting is off); any pointer may be NULL. */
PIC_API int pic_count_lifts(pic_t h, int32_t enable);
PIC_API int pic_lift_counts(pic_t h, int64_t *lifts, int64_t *drops, int64_t *tunnellers, int64_t *steps);

/* Phases of a step for pic_phase_times. */
#define PIC_PHASE_DEPOSIT 0  /* leaf partial sums + vertex charges + FP64 total */
#define PIC_PHASE_SOLVE 1    /* built-in Jacobi sweeps + vertex field (or the hook) */
#define PIC_PHASE_PUSH 2     /* fused gather + push + re-location + key + counts */
#define PIC_PHASE_REBIN 3    /* offsets scan, stayer ranks, mover compaction + slots */
#define PIC_PHASE_PERMUTE 4  /* permutation of the particle arrays into bucket order */
#define PIC_NPHASES 5

/* Diagnostics without a counterpart in the paper.  Per-phase device timing
 * with CUDA events recorded on the handle's stream
 * around every phase of every later call.  enable = 0 stops recording;
 * enable = 1 (re)starts it from zero. */
PIC_API int pic_profile(pic_t h, int32_t enable);

/* Synchronises the stream and returns, per phase, the summed device time in
 * milliseconds and the number of this library's kernels launched, since the
 * last pic_profile(h, 1).  Both arrays have PIC_NPHASES entries. */
PIC_API int pic_phase_times(pic_t h, double *ms, int64_t *kernels);

/* Tables of the spacetree (Section 4), its finite-element grid (Section 3)
 * and dual tree (Section 4.1), for tests: leaf level[n_leaves] and
 * coords[n_leaves][d]; vertex
 * positions pos[d][n_vertices] in units of 3^-depth; PIDT owner vertices
 * level[n_buckets], j[n_buckets][d] (host memory; PIDT handles only, else
 * PIC_ESTATE). */
PIC_API int pic_leaf_table(pic_t h, int32_t *level, int64_t *coords);
PIC_API int pic_vertex_table(pic_t h, int64_t *pos);
PIC_API int pic_pidt_table(pic_t h, int32_t *level, int64_t *j);
/* The finite-element tables of a single-instance handle with an adaptive tree
 * (Section 3 grid on the Section 4 tree; PIC_ESTATE otherwise), as the
 * kernels read them, for tests: every leaf corner expanded onto vertices,
 * cexp_ptr[n_leaves 2^d + 1], cexp_vid[*n_entries], cexp_w[*n_entries], and
 * per vertex ion_load[n_vertices] and diag[n_vertices] (host memory; any
 * pointer may be NULL; pass NULL arrays first to learn *n_entries).  The
 * layout is that of pic_tree_tabulate. */
PIC_API int pic_grid_tables(pic_t h, int64_t *n_entries, int32_t *cexp_ptr, int32_t *cexp_vid, double *cexp_w,
                            double *ion_load, double *diag);

/* Replace the tree (same d) and re-bin the particles into it: the dynamic
 * adaptivity of Section 5's introduction (the grid changes between steps and
 * every particle is lifted and dropped into the leaf or dual cell of the new
 * grid that covers it; Theorems 1 and 2 hold for any tree).  FP64 particles
 * keep their positions; split particles are re-located with the integer
 * lift/drop rule of the split push (zero displacement).  The solver's warm
 * start and the field are reset.  Malformed tree or other d: PIC_EINVAL.
 * Synchronous. */
PIC_API int pic_retree(pic_t h, const pic_tree_desc *tree);

/* The raPIDT tree attribute v_max (Section 5.4, the v_max equation): per node
 * of the tree, in the level order of its refinement flags, the largest
 * velocity component magnitude of the particles below it -- on a leaf, of its
 * own particles (PIT) or of the particles of its 2^d vertices, i.e. of every
 * dual cell intersecting it (PIDT); on a refined cell, the largest of its
 * children's values.  node_vmax[n_nodes] (host memory, may be NULL);
 * *n_closed (may be NULL) = the nodes with v_max dt < 3^-level, from which no
 * particle can be removed by a lift within a step of dt.  Computed from the
 * current particles on the device; synchronous; single-instance handles only
 * (PIC_ESTATE otherwise). */
PIC_API int pic_vmax(pic_t h, double *node_vmax, double dt, int64_t *n_closed);

/* Level-order refinement flags of the current spacetree (Section 4; the
 * encoding of pic_tree_desc): with flags == NULL only *n_nodes is written;
 * else flags[n_nodes] (host memory). */
PIC_API int pic_tree_flags(pic_t h, uint8_t *flags, int64_t *n_nodes);

/* ---- checkpoint / resume ----------------------------------------------------
 * The paper has no counterpart to these calls: they are library utilities.
 * pic_save writes what the next step reads: the refinement flags of every
 * instance, the particle state in storage order and native precision (split:
 * leaf ids, FP32 offsets, FP32 velocities; FP64: positions, velocities), the
 * particle ids (track_ids), the potential V (the warm start of the built-in
 * solve), the field E, the step counter, the configuration (everything in
 * pic_config but the stream) and the launch tuning.  Velocities are saved as
 * they are, so a leapfrog run resumes at its half step.  Synchronous; the file
 * is overwritten.  PIC_ESTATE if the handle holds a sticky device error,
 * PIC_EIO if the file cannot be written.
 *
 * pic_load creates a new handle (*out, on `stream`) from such a file.  Steps
 * of the loaded handle give the same bits as steps of the saved one: sort
 * keys, bucket offsets and vertex charges are recomputed from the saved
 * state, which stays in its saved order.  PIC_EIO: the file is missing,
 * unreadable, not a checkpoint, of another format version, truncated, or its
 * checksum does not match.  PIC_EINVAL: its trees are malformed or a particle
 * value is out of range (a non-finite value, an offset or FP64 position
 * outside [0, 1), a leaf outside the particle's instance, ids that are not a
 * permutation of [0, n)).  Every such check runs on the host before the first
 * device call.  On failure *out is NULL and pic_last_error(NULL) says why.
 *
 * File layout (little-endian; each section zero-padded to 8 bytes):
 *   magic "PICSNAP\0", u32 version 1, u32 meta bytes, u64 checksum of all
 *   bytes after these 24; meta: i32 d, scheme, precision, sweeps, track_ids,
 *   path, n_inst, 0; f64 q, qm, ion, omega; i64 step, n, n_vertices;
 *   i32 tuning[4]; per instance i64 n_flags, i64 n_particles, f64 q; then
 *   flags u8[], leaf i32[n] (split only), pos[d][n], vel[d][n] (f32 split,
 *   f64 otherwise), ids i32[n] (track_ids only), V[n_vertices],
 *   E[d][n_vertices].  The checksum folds the 64-bit words w in order:
 *   c = 0x243f6a8885a308d3 initially, then c = (c ^ w) * 0x9e3779b97f4a7c15
 *   and c ^= c >> 29 (arithmetic mod 2^64). */
PIC_API int pic_save(pic_t h, const char *path);
PIC_API int pic_load(pic_t *out, const char *path, void *stream);

/* Re-refine by the particles-per-cell criterion: cell C on level m is refined
 * iff m < dmin, or m < dmax and C holds more than ppc particles (Section 6
 * setup: refine on overrun, coarsen when the union stays within ppc).  Counts
 * per level are taken on the device; dmax <= 6 in 3D, <= 10 in 2D.  Split
 * positions below their leaf are resolved with the drop rule.  A resulting
 * tree equal to the current one keeps every bucket (only the solver's warm
 * start and the field are reset, as by pic_retree); any other is installed by
 * pic_retree.  Synchronous. */
PIC_API int pic_adapt(pic_t h, int64_t ppc, int32_t dmin, int32_t dmax);

/* ---- no-allocation entry point -------------------------------------------
 * The paper has no counterpart to this call: it is a library utility.  It is
 * the stable counting sort of the re-bin (Section 4) for the fresh-particle
 * case, on caller-owned device keys, for callers that must not allocate
 * device memory at that point: a thread that runs while another thread holds
 * a global-mode stream capture (cudaMalloc is refused there), a pipeline
 * that cannot afford cudaFree's implicit device synchronisation between
 * steps, or a process whose memory a caching allocator has already reserved.
 *
 * keys[n] (device): bucket of each element, in [0, n_keys).  Outputs (device,
 * caller-owned, no initialisation needed): start[n_keys + 1] exclusive bucket
 * offsets, start[n_keys] = number of valid keys; perm[n] the input index at
 * each sorted position, ascending inside every bucket (stable).  Keys outside
 * [0, n_keys) are skipped, so start[n_keys] < n reports them and perm past
 * start[n_keys] is left untouched.
 *
 * Work is queued on `stream` (a cudaStream_t; NULL = legacy default stream)
 * and the call returns without synchronising.  Scratch is one file-scope
 * device array of PIC_NOALLOC_MAX_KEYS + 192 int32 words per device
 * (4 MiB); the call clears the part it uses on `stream`, so nothing must be
 * zero on entry.  No device memory is allocated or freed.  That array is
 * shared by every caller in the process: calls on one device that overlap in
 * time (different streams or host threads) race and must be serialised by
 * the caller.  The first call on each device looks the array's address up
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call outside any stream capture, and make no call on a device after
 * cudaDeviceReset() on it (the module, and with it the array, is reloaded at
 * another address).  No statement is made about capturing later calls in a
 * CUDA graph.  Crowded buckets cost O(m log^2 m) for a bucket of m elements.
 *
 * Returns PIC_EINVAL for n < 0, n > INT32_MAX, n_keys < 1, NULL pointers, or
 * n_keys > PIC_NOALLOC_MAX_KEYS (nothing is launched); PIC_ECUDA if a CUDA
 * call fails. */
#define PIC_NOALLOC_MAX_KEYS (1 << 20)
PIC_API int pic_bucket_noalloc(const int32_t *keys, int64_t n, int64_t n_keys, int32_t *start, int32_t *perm,
                               void *stream);

/* Host-only tabulation of a spacetree given as level-order refinement flags
 * (Section 4: the tree, its d-linear finite-element grid with hanging-vertex
 * constraints, and the PIDT owner vertices), without a handle and without
 * any device work, so it can run where there is no GPU.  Call once with
 * every array NULL to learn the sizes, then again with caller-owned host
 * arrays of those sizes; any array may be NULL.
 *   vertex_pos[d][n_vertices]   non-hanging vertices in units of 3^-depth
 *   pidt_level[n_pidt_vertices], pidt_j[n_pidt_vertices][d]  PIDT owners
 * and, for trees that are not uniform (sizes->uniform == 0; uniform trees
 * use closed forms and leave these untouched):
 *   ion_load[n_vertices], diag[n_vertices]  load of a unit density and the
 *                                           stiffness diagonal per vertex
 *   cexp_ptr[n_leaves 2^d + 1], cexp_vid[n_corner_entries],
 *   cexp_w[n_corner_entries]    every leaf corner expanded onto vertices
 * Returns PIC_EINVAL for a NULL sizes pointer or a malformed tree. */
typedef struct {
  int32_t d, depth, uniform, reserved;
  int64_t n_leaves, n_vertices, n_corner_entries, n_pidt_vertices;
} pic_tree_sizes_t;
PIC_API int pic_tree_tabulate(int32_t d, const uint8_t *flags, int64_t n_flags, pic_tree_sizes_t *sizes,
                              int64_t *vertex_pos, double *ion_load, double *diag, int32_t *cexp_ptr,
                              int32_t *cexp_vid, double *cexp_w, int32_t *pidt_level, int64_t *pidt_j);

/* Stream-like particle update, the calibration ceiling of the paper's
 * memory-throughput experiment (Section 6, "Memory throughput"): `steps`
 * passes over the particles, each advancing every position by one explicit
 * Euler step x += v dt and reflecting it at the walls of the unit box
 * (x < 0 -> -x, x > 1 -> 2 - x, the velocity component negated), written back
 * in place.  No grid, no keys, no reordering.  Not part of the particle step:
 * it bounds what a particle update can reach on the same memory system.
 *
 * d = 2 or 3; precision PIC_FP64 (double arrays) or PIC_FP32_SPLIT (float
 * arrays, FP32 arithmetic with separate roundings of the product and the
 * sum); x[d][n] and v[d][n] are device arrays, structure of arrays, owned by
 * the caller and updated in place.  Work is queued on `stream` (a
 * cudaStream_t; NULL = legacy default stream), one kernel per pass; the call
 * does not synchronise.  Returns PIC_EINVAL for a bad d, precision, n < 0,
 * steps < 0 or NULL arrays with n > 0; PIC_ECUDA if a launch fails. */
PIC_API int pic_stream_step(int32_t d, int32_t precision, void *x, void *v, int64_t n, double dt, int32_t steps,
                            void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PIC_H */
