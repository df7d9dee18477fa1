/*
 * lvb.h -- C-ABI of liblvb, a GB300 (sm_103a) local Verlet buffer broad
 * phase for soft-sphere DEM, after "Local Verlet buffer approach for
 * broad-phase interaction detection in Discrete Element Method"
 * (arXiv 2208.13770).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Particle arrays are float4 records in structure-of-arrays form, passed
 *   as `const float*` to 16-byte-aligned DEVICE memory:
 *     pos_r : (x, y, z, r)          position [m] and radius [m]
 *     vel   : (vx, vy, vz, unused)  velocity [m/s]
 *     acc   : (ax, ay, az, unused)  acceleration [m/s^2]
 *   n records each, particle i at float offset 4*i.
 * - Output buffers of the lvb_get_* / dem_get_* calls may be host or device
 *   memory: the library copies into them with cudaMemcpyDefault (unified
 *   addressing tells the two apart).  The caller owns every buffer it passes; the library never
 *   keeps a caller pointer beyond the call.
 * - All work is enqueued on the context's CUDA stream (`void* stream` is a
 *   cudaStream_t; NULL is the legacy default stream).  Calls that only
 *   enqueue return before the GPU finishes; caller buffers must stay valid
 *   until the stream reaches that point.
 * - Return value: 0 (LVB_OK) or a negative LVB_E* code; no exception, exit
 *   or device trap crosses this boundary.  Errors found on the device (a
 *   non-finite position, a full cell, a full pair store) are sticky: they
 *   are returned by lvb_sync and by every later call that synchronises
 *   (the lvb_get_* family, lvb_stats), and the context's list is invalid
 *   from the step that raised them on.
 * - A context is not thread-safe; distinct contexts are independent.
 *
 * Definitions (binary32, round to nearest, no fused multiply-add):
 *   |a - b|^2 = ((dx*dx + dy*dy) + dz*dz) with d = a - b per component.
 *   R_NL,i    = r_i + skin_i                            (Eq. bounding_sphere)
 *   flag_i    : |x_i - xref_i|^2 > skin_i * skin_i    (Eq. update; xref_i is
 *               the position of i at its last list update)
 *   pair {i,j}: |xref_i - xref_j|^2 <= (R_NL,i + R_NL,j)^2
 *               (Def. verletlist and Eq. broad_phase, on reference positions)
 *   contact   : delta_ij = (r_i + r_j) - sqrt(|x_i - x_j|^2) > 0 (Eq. delta)
 */
#ifndef LVB_H
#define LVB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LVB_OK          0
#define LVB_EINVAL     (-1)  /* bad argument (NULL, n <= 0, misaligned, bad enum, box) */
#define LVB_ENOMEM     (-2)  /* device allocation failed */
#define LVB_ECAPACITY  (-3)  /* caller's output buffer too small: the needed
                                size is written to the count argument */
#define LVB_EDEVICE    (-4)  /* a CUDA call failed */
#define LVB_ENAN       (-5)  /* a non-finite position or radius was seen */
#define LVB_EOVERFLOW  (-6)  /* an internal fixed-capacity store overflowed
                                (cell slots or pair store); list invalid */
#define LVB_ESTATE     (-7)  /* call not valid in the context's state */
#define LVB_ELIMIT     (-8)  /* input larger than a fixed-size entry point's
                                stated maximum (lvb_noalloc.h) */
#define LVB_ETIMEOUT   (-9)  /* a grid-wide barrier of the step kernel waited
                                past its limit (about a second); the step was
                                abandoned and the context is unusable */

/* Skin policies (Sec. "The local skin parameter" and Sec. Results). */
#define LVB_SKIN_GLOBAL           0  /* skin = value (uniform; the paper's
                                        constant-skin comparator) */
#define LVB_SKIN_DIAMETER_FACTOR  1  /* skin = value * (2 r_i) */
#define LVB_SKIN_PAPER_KVDT       2  /* skin = (value * |v_i|) * dt with
                                        value = K, Eq. skin_formulus1 */
#define LVB_SKIN_LEARNED          3  /* skin proposed by the skin network
                                        (lvb_mlp.h); needs vel and acc */

/* When the list is updated (Def. autoverlet and its per-particle form). */
#define LVB_TRIGGER_PARTIAL 0  /* only flagged particles update xref/skin and
                                  get their rows rebuilt (local buffer) */
#define LVB_TRIGGER_GLOBAL  1  /* any flag => every particle updates and the
                                  whole list is rebuilt (Def. autoverlet) */
#define LVB_TRIGGER_ALWAYS  2  /* every step is a full rebuild ("without
                                  Verlet buffer" when the skin is 0) */

typedef struct lvb_ctx lvb_ctx;

typedef struct {
    int32_t kind;        /* LVB_SKIN_* */
    float value;         /* s_g [m], alpha [-] or K [steps], by kind */
    float dt;            /* time step for LVB_SKIN_PAPER_KVDT [s] */
    const void *mlp;     /* LVB_SKIN_LEARNED: device pointer to packed
                            weights (lvb_mlp.h layout), 16-byte aligned;
                            else NULL */
} lvb_skin_policy;

typedef struct {
    float lo[3];         /* box lower corner [m] */
    float hi[3];         /* box upper corner [m]; hi > lo per axis */
} lvb_box;

typedef struct {
    int64_t n;               /* particles */
    int64_t steps;           /* lvb_step calls completed */
    int64_t rebuild_steps;   /* steps at which at least one particle updated */
    int64_t flagged_total;   /* sum over steps of |flagged| */
    int64_t updated_total;   /* sum over steps of particles whose xref/skin
                                were updated (= flagged_total in PARTIAL mode) */
    int64_t last_flagged;    /* |flagged| at the last step */
    int64_t entries;         /* symmetric list entries (2 x pairs) */
    int64_t pairs;           /* unordered pairs in the list */
    int64_t relayouts;       /* row-store re-layouts (a row outgrew its slack) */
    int64_t grows;           /* times the row store or the cell slots grew */
    int64_t cell_capacity;   /* slots per cell */
    int64_t row_store_capacity; /* entries the row store can hold */
    int64_t kernels_executed;  /* kernels of this context run on the device
                                  (including the DEM driver's, if any) */
    int64_t barriers;        /* grid-wide barriers passed by step kernels */
    int64_t step_blocks;     /* blocks of the step kernel (all resident) */
    int64_t block_threads;   /* threads per block of the step kernel */
    int64_t compaction;      /* LVB_COMPACT_* in use */
    int64_t n_scenes;        /* independent scenes in the context */
    /* work of the partial rebuilds so far (PARTIAL trigger), the counts
     * behind the algorithmic bytes of a step: */
    int64_t rebuild_candidates; /* stencil candidates read (cell slot id +
                                   reference record each) */
    int64_t rebuild_direct;  /* flagged-list records read by the direct test
                                of the flagged particles against each other */
    int64_t rebuild_edits;   /* edits of unflagged particles' rows (a pair
                                removed or inserted) */
    int64_t reserved[1];
    float cell_edge;         /* L [m] (scene 0) */
    float rnl_max;           /* cap H on R_NL = r + skin [m] (scene 0) */
    int32_t grid[3];         /* cells per axis (scene 0) */
    int32_t pad;
} lvb_stats_t;

typedef struct {
    int64_t first;           /* first particle of the scene */
    int64_t count;           /* particles of the scene */
    float cell_edge;         /* L [m] */
    float rnl_max;           /* cap H on R_NL = r + skin [m] */
    int32_t grid[3];         /* cells per axis */
    int32_t pad;
} lvb_scene_info_t;

/*
 * lvb_init -- build the context and the first list (Algorithm 1 on the
 * extended spheres) at the given positions, which become every particle's
 * reference position.
 *
 *   out         : receives the context.
 *   n           : particles, 1 <= n < 2^31.
 *   pos_r       : device float4 (x, y, z, r), n records; radii are read
 *                 here and kept fixed for the life of the context.
 *   box         : the domain.  Positions outside it are binned into the
 *                 boundary cells (correct, but slow if many leave it).
 *   skin        : skin policy.
 *   trigger     : LVB_TRIGGER_*.
 *   cell_factor : cell edge L = cell_factor * (largest diameter)
 *                 * (1 + 2^-7), cell_factor >= 1.  Every skin is capped so
 *                 that R_NL <= H = L/2 * (1 - 2^-8) (the cap of Eq.
 *                 skin_formulus_mincell, read as R_NL bounded by half a
 *                 cell so the 27-cell stencil sees every pair).
 *   vel         : device float4 velocities, needed by LVB_SKIN_PAPER_KVDT
 *                 and LVB_SKIN_LEARNED; may be NULL otherwise.
 *   acc         : device float4 accelerations, needed by LVB_SKIN_LEARNED;
 *                 may be NULL otherwise.
 *   stream      : cudaStream_t for all work of this context.
 * Synchronises the stream.  Errors: EINVAL, ENOMEM, ENAN, EDEVICE.
 */
int lvb_init(lvb_ctx **out, int64_t n, const float *pos_r, const lvb_box *box,
             const lvb_skin_policy *skin, int32_t trigger, float cell_factor,
             const float *vel, const float *acc, void *stream);

/*
 * lvb_batch_init -- one context over n_scenes independent scenes that
 * advance together: scene s is particles [offsets[s], offsets[s+1]) of the
 * arrays, with its own box boxes[s] and its own cell grid (edge from the
 * scene's largest diameter), and no pair ever joins two scenes.  Every step
 * of the context covers all scenes in the same launches, so many small
 * scenes run at the throughput of one large one.
 *   offsets : host, n_scenes + 1 entries, offsets[0] = 0, strictly
 *             increasing, offsets[n_scenes] = total particles.
 *   boxes   : host, n_scenes boxes.
 * Other arguments as lvb_init.  The GLOBAL trigger is per context, so it is
 * rejected (EINVAL) for n_scenes > 1; PARTIAL and ALWAYS are per particle.
 */
int lvb_batch_init(lvb_ctx **out, int32_t n_scenes, const int64_t *offsets,
                   const float *pos_r, const lvb_box *boxes, const lvb_skin_policy *skin,
                   int32_t trigger, float cell_factor, const float *vel, const float *acc,
                   void *stream);

/* lvb_scene_info -- geometry of one scene of a context. */
int lvb_scene_info(lvb_ctx *ctx, int32_t scene, lvb_scene_info_t *out);

/*
 * lvb_init_resume -- as lvb_init, but every particle's reference state is
 * taken from ref4 (device float4 (xref, yref, zref, skin), n records, e.g.
 * saved by lvb_get_ref) instead of being set from pos_r and the policy;
 * pos_r still supplies the radii.  The list is built on those references,
 * so a run resumes exactly where the saved context stood (the list is a
 * function of the reference state alone, Def. verletlist).  Each skin must
 * be finite, >= 0 and within the cap max(0, H - r) of the new context, else
 * LVB_EINVAL.
 */
int lvb_init_resume(lvb_ctx **out, int64_t n, const float *pos_r, const float *ref4,
                    const lvb_box *box, const lvb_skin_policy *skin, int32_t trigger,
                    float cell_factor, const float *vel, const float *acc, void *stream);

/*
 * lvb_batch_init_resume -- lvb_batch_init with every particle's reference
 * state taken from ref4 (device float4 (xref, yref, zref, skin), n records,
 * e.g. saved by lvb_get_ref of a batched context), as lvb_init_resume does
 * for one scene: the list of each scene is built on those references, so a
 * batched run resumes where the saved context stood.  Same checks as
 * lvb_init_resume (each skin within the cap of its own scene, else
 * LVB_EINVAL) and as lvb_batch_init.
 */
int lvb_batch_init_resume(lvb_ctx **out, int32_t n_scenes, const int64_t *offsets,
                          const float *pos_r, const float *ref4, const lvb_box *boxes,
                          const lvb_skin_policy *skin, int32_t trigger, float cell_factor,
                          const float *vel, const float *acc, void *stream);

/*
 * lvb_step -- one step of the automatic Verlet update at the positions
 * pos_r (same n and radii as at init), as one cooperative kernel launch:
 *   1. flag every particle whose displacement since its reference position
 *      exceeds its skin (Eq. update);
 *   2. update reference position and skin of the flagged particles
 *      (PARTIAL), of all particles if any is flagged (GLOBAL), or of all
 *      (ALWAYS);
 *   3. re-bin the updated particles in the linked-cell grid and rebuild
 *      exactly the list rows that change.
 * After the step the list equals the pair set defined above on the current
 * (xref, skin) of all particles.  vel/acc as for lvb_init.
 * Enqueues only (no synchronisation).  Errors: EINVAL, EDEVICE; device-side
 * errors are reported by lvb_sync.
 */
int lvb_step(lvb_ctx *ctx, const float *pos_r, const float *vel, const float *acc);

/*
 * lvb_step_host -- lvb_step with its inputs in host memory and the step's
 * flags returned to host memory (the same step as lvb_step).
 *   pos_r, vel, acc : host, n x 4 float as for lvb_step (vel / acc NULL
 *                     unless the skin policy needs them).
 *   bits            : host, ceil(n / 32) words out: the flag bits of this
 *                     step (bit i % 32 of word i / 32); may be NULL.
 *   n_flagged       : host, one int out: particles flagged at this step;
 *                     may be NULL.
 * Enqueues only.  The inputs are copied into one of two device staging
 * slots owned by the context, on a copy stream of its own, so the copy of a
 * step's inputs overlaps the previous step's kernel; the step waits for its
 * copy and writes its flags also into the slot, which a second copy stream
 * of the context copies out to `bits` / `n_flagged` while the next step
 * runs.
 * Every host buffer must stay valid, and the inputs unchanged, until
 * lvb_sync (or another synchronising call) returns.  Page-locked host
 * memory (cudaHostAlloc, cudaHostRegister) lets the copies overlap; with
 * pageable memory the results are the same but the copies serialise.  The
 * staging slots are allocated on the first call (2 x n x 16 bytes per
 * input given, and 2 x (ceil(n / 32) + 1) x 4 bytes for the outputs).
 * Errors: EINVAL (as lvb_step), ENOMEM, EDEVICE.
 */
int lvb_step_host(lvb_ctx *ctx, const float *pos_r, const float *vel, const float *acc,
                  uint32_t *bits, int32_t *n_flagged);

/* Options of lvb_set_option.  None of them changes a result. */
#define LVB_OPT_TRACE     3  /* 1: the step kernel records the device time of
                                its phases, the DEM driver's separate kernels
                                theirs, read with lvb_trace; 0 (default): off */
#define LVB_OPT_BLOCK_THREADS 4 /* block size of the step kernel: 1024
                                (default, one block per SM), 512 or 256
                                (two or four per SM) */
#define LVB_OPT_COMPACT   5  /* compaction of the flagged ids in the check:
                                LVB_COMPACT_WARP (default) or LVB_COMPACT_BLOCK */
/* Failure test hooks (the grid-wide barrier's bounded wait): */
#define LVB_OPT_BARRIER_EXTRA 6 /* 1: every barrier waits for one arrival more
                                than the grid has, so the next step's wait
                                runs out: the step is abandoned and the
                                context reports LVB_ETIMEOUT (as after a
                                real stall); 0 (default): normal */
#define LVB_OPT_BARRIER_SPINS 7 /* polls (L2 round trips) before a barrier gives
                                up, 1 .. 2^22 (default 2^22, about a second or
                                two) */
#define LVB_OPT_DIRECT_MAX 8  /* largest flagged count whose rebuild runs in one
                                phase (cell moves and rows together, flagged
                                pairs found by a direct test of the flagged
                                particles against each other); above it the
                                moves come first, then a barrier, then the
                                rows from the final cells.  0 .. 2^20
                                (default 4096) */

#define LVB_OPT_STENCIL_REACH 9 /* which of the 27 stencil cells a row build
                                scans (Algorithm 1 visits all 27): 0 all of
                                them; 1 those whose box lies within R_NL,i + H
                                of the particle (H the cap on any R_NL); 2
                                (default) also skips a cell whose box lies
                                beyond R_NL,i plus the largest R_NL stored in
                                that cell.  Every partner lies within
                                R_NL,i + R_NL,j, so each choice gives the same
                                list; 1 and 2 read fewer candidates with
                                polydisperse radii */

#define LVB_OPT_CELL_CAPACITY 12 /* slots per cell of at least value (rounded
                                up to a multiple of 32, at most 65536): the
                                cells are re-laid out before the next step
                                (no effect if they already have as many).
                                The library sizes the slots from the initial
                                occupancy and a dense packing of the mean
                                particle volume, and doubles them between
                                steps when a cell passes 75%; a caller that
                                moves many particles into one cell within
                                one step raises them first */

#define LVB_OPT_HISTORY 13  /* 1: keep one contact-history record (4 floats)
                                beside every list entry: a partial rebuild
                                edits a flagged particle's row in place, so
                                every partner that stays a pair keeps its
                                slot and record, a new pair's record starts
                                at zero, and re-layouts and store growth
                                carry each record to the entry's new slot
                                (the DEM driver's tangential springs live
                                there).  PARTIAL trigger only (else
                                LVB_EINVAL); the lists are the same as
                                without it.  0 (default): off */

/* Test hooks for the overflow paths (they make a store fill up without a
 * device fault; the results of a context that reports LVB_EOVERFLOW are
 * invalid, as always): */
#define LVB_OPT_GROW 10       /* 1 (default): the host grows the cell slots and
                                the row store between steps when a kernel
                                finds them over 75% / 60% full; 0: requests
                                are ignored, so a cell that fills up reports
                                LVB_EOVERFLOW */
#define LVB_OPT_FORCE_RELAYOUT 14 /* 1: the next step that rebuilds rows
                                re-lays out the whole row store on the device
                                as if a row had outgrown its slack (test hook
                                for the re-layout path; the list is the same) */
#define LVB_OPT_STORE_LIMIT 11 /* entries of the row store a re-layout may use:
                                0 (default) the whole allocation, else
                                min(value, allocation); a re-layout that does
                                not fit even without slack reports
                                LVB_EOVERFLOW */

#define LVB_OPT_EARLY 16      /* the early trigger, beta = value / 1000 (as
                                binary32), 1 .. 1000 (1000, the default: off).
                                On a step where some particle violates Eq.
                                update, every particle with |x - xref|^2 >
                                (beta skin)^2 (binary32: t = beta * skin,
                                then t * t) is updated with it, so the next
                                violation comes later and fewer steps pay a
                                rebuild.  The list stays the pair set of the
                                reference states; lvb_get_flags still returns
                                the violations, lvb_stats counts both.  One
                                scene, PARTIAL trigger (else LVB_EINVAL) */
#define LVB_OPT_CHECK_LOADS 15 /* how the displacement check of lvb_step reads
                                pos and ref: LVB_CHECK_REGS (default) or
                                LVB_CHECK_RING */

/* Values of LVB_OPT_CHECK_LOADS. */
#define LVB_CHECK_REGS 1     /* each warp loads four chunks of 32 particles
                                into registers at once (streaming loads) */
#define LVB_CHECK_RING 0     /* thread 0 of each block streams tiles through
                                a four-stage shared-memory ring of bulk copies */

/* Values of LVB_OPT_COMPACT. */
#define LVB_COMPACT_WARP  0  /* flagged ids gather in a per-warp list during
                                the check; the list takes its indices with
                                one atomic per warp when it fills and at the
                                end of the check */
#define LVB_COMPACT_BLOCK 1  /* the same, but at the end of the check the
                                warps' lists take their indices together,
                                with one atomic per block after a block scan
                                (two block barriers) */

/* Slots of lvb_trace. */
#define LVB_TRACE_SLOTS 16
/* Phases of the step kernel: 0 check (with the flagged particles'
 * updates), 1 rebuild passes, 2 re-layout, 3 tail (the DEM driver's
 * forces); separate kernels: 4 DEM integrate, 5 DEM forces, 6 full-build
 * rows (init, store growth); inside the partial rebuild: 7 from the first
 * work item's start to the last one's end (patches and moves), 8 the
 * longest single work item. */

/* lvb_trace -- per-kernel device time summed over the steps traced so far
 * (ns) and the number of steps each kernel ran in; LVB_TRACE_SLOTS entries
 * each.  Synchronises. */
int lvb_trace(lvb_ctx *ctx, uint64_t *sum_ns, uint64_t *count);

/* lvb_set_option -- set an LVB_OPT_* value (synchronises if a cached graph
 * has to be rebuilt).  Errors: EINVAL. */
int lvb_set_option(lvb_ctx *ctx, int32_t option, int64_t value);

/* lvb_sync -- wait for the context's stream and return the sticky device
 * error (LVB_OK, LVB_ENAN, LVB_EOVERFLOW or LVB_ETIMEOUT). */
int lvb_sync(lvb_ctx *ctx);

/*
 * lvb_get_pairs -- the list as a compacted symmetric CSR: row i holds every
 * j with {i, j} in the list, ascending; row_ptr has n + 1 entries.
 * cap is the capacity of col.  If the list has more entries than cap,
 * returns LVB_ECAPACITY with *n_entries set and row_ptr filled.
 * Synchronises.
 */
int lvb_get_pairs(lvb_ctx *ctx, int32_t *row_ptr, int32_t *col, int64_t cap,
                  int64_t *n_entries);

/* lvb_get_pairs_ij -- the list as unordered pairs i < j, sorted by (i, j).
 * Same capacity rule as lvb_get_pairs.  Synchronises. */
int lvb_get_pairs_ij(lvb_ctx *ctx, int32_t *pi, int32_t *pj, int64_t cap,
                     int64_t *n_pairs);

/*
 * lvb_get_near_cutoff -- the pairs i < j, in the list or not, whose squared
 * reference distance d2 (the fixed binary32 formula of the definitions
 * above, Def. verletlist) lies within a relative distance rel of their
 * squared cutoff c2 = (R_NL,i + R_NL,j)^2 (binary32): |d2 - c2| <= rel c2,
 * compared in binary64 from the two binary32 values.  These are the pairs
 * whose membership rests on the last bits of the formula; they are listed
 * apart from the list so that a comparison with another evaluation can
 * tell a rounding difference from an error.
 *   rel             : 0 <= rel <= 2^-8 (e.g. 1e-6); every such pair lies in
 *                     the 27 cells around either particle's cell.
 *   pi, pj          : host or device int32 out, cap entries each, in no
 *                     particular order.
 *   n_pairs         : out, the number of such pairs.
 * Synchronises.  Errors: EINVAL, ECAPACITY (count written to *n_pairs),
 * EDEVICE, and the context's device errors.
 */
int lvb_get_near_cutoff(lvb_ctx *ctx, double rel, int32_t *pi, int32_t *pj, int64_t cap,
                        int64_t *n_pairs);

/*
 * lvb_get_contacts -- narrow phase (Eq. delta) on the list at positions
 * pos_r: every pair i < j of the list with delta_ij > 0, sorted by (i, j),
 * with delta_ij (binary32 formula above).  Same capacity rule.
 * Synchronises.
 */
int lvb_get_contacts(lvb_ctx *ctx, const float *pos_r, int32_t *ci, int32_t *cj,
                     float *delta, int64_t cap, int64_t *n_contacts);

/* lvb_get_flags -- flags of the last step as a bitmask, bit (i % 32) of
 * word i / 32; ceil(n/32) words.  *n_flagged = number of set bits.
 * Synchronises. */
int lvb_get_flags(lvb_ctx *ctx, uint32_t *bits, int64_t *n_flagged);

/* lvb_get_ref -- per-particle reference state (xref, yref, zref, skin),
 * n float4 records.  Synchronises. */
int lvb_get_ref(lvb_ctx *ctx, float *ref4);

/* lvb_stats -- counters and geometry of the context.  Synchronises. */
int lvb_stats(lvb_ctx *ctx, lvb_stats_t *out);

/* lvb_set_stream -- move the context to another stream (no copy). */
int lvb_set_stream(lvb_ctx *ctx, void *stream);

/* lvb_destroy -- free the context (synchronises its stream first). */
int lvb_destroy(lvb_ctx *ctx);

/* lvb_strerror -- static description of a status code. */
const char *lvb_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* LVB_H */
