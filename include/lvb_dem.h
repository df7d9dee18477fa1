/*
 * lvb_dem.h -- C-ABI of the DEM driver that runs on top of the local Verlet
 * buffer broad phase (lvb.h): velocity Verlet integration and a normal-only
 * linear spring-dashpot contact law, with the contact search on the list.
 *
 * The paper's runs use velocity Verlet and a linear spring-dashpot model
 * (Sec. Methodology); the loop is its XDEM flow chart with the list-validity
 * gate before the broad phase (Sec. "XDEM flow chart", Fig.
 * xdemw_flow_chart): integrate, broad phase (skipped per particle while its
 * list rows stay valid), narrow phase on the list, forces, integrate.
 *
 * One step, with state (x, v, a) on the device (binary32):
 *   x'  = x + v dt + a dt^2 / 2            (positions; then the broad phase
 *   v*  = v + a dt                           runs at x', with v* as the
 *                                            velocity seen by the skin rule)
 *   F   = sum over list partners j with delta_ij > 0 of
 *         (k_n delta_ij - gamma_ij v_n,ij) n_ij, plus walls
 *         delta_ij = r_i + r_j - |x'_i - x'_j|   (Eq. delta; evaluated with
 *                    compensated binary32 arithmetic, error ~1e-16 m)
 *         n_ij = (x'_i - x'_j)/|x'_i - x'_j|, v_n,ij = (v*_i - v*_j) . n_ij
 *         gamma_ij = 2 zeta sqrt(m_eff k_n), zeta = -ln e / sqrt(pi^2+ln^2 e),
 *         m_eff = m_i m_j / (m_i + m_j), m = rho 4/3 pi r^3
 *   a'  = F/m + g,   v' = v + (a + a') dt / 2
 * With friction (mu > 0; the paper's LSD model with static friction, Sec.
 * Methodology) each particle also carries an angular velocity w (moment of
 * inertia I = 2/5 m r^2, velocity Verlet as for v: w* = w + al dt, w' = w +
 * (al + al') dt / 2) and each contact a tangential spring xi, kept in the
 * broad phase's contact history (LVB_OPT_HISTORY), so it survives partial
 * rebuilds:
 *   v_rel = (v*_i - v*_j) - (r_i w*_i + r_j w*_j) x n_ij   (contact point)
 *   v_t   = v_rel - (v_rel . n_ij) n_ij
 *   xi    = xi - (xi . n_ij) n_ij,  then xi = xi + v_t dt
 *   F_t   = -k_t xi - gamma_t v_t, capped at mu max(F_n, 0) (then
 *           xi = -(F_t + gamma_t v_t) / k_t)
 *   force on i: F_n n_ij + F_t;  torque on i: -r_i n_ij x F_t
 * A pair out of contact has xi = 0; both sides of a pair keep exactly
 * opposite records (the same binary32 operations with the roles swapped).
 * Walls use the same law with m_eff = m_i: box planes (wall_kind 1), a drum
 * of radius R about the y axis through (drum_cx, drum_cz) with end caps at
 * the box's y planes (kind 2; the wall moves tangentially, which a normal-
 * only law does not see), or specular reflection at the box planes (kind 3,
 * meant for runs without contacts or gravity).
 *
 * Pointers follow lvb.h: device float4 records in, host or device buffers
 * out, errors as LVB_* codes.
 */
#ifndef LVB_DEM_H
#define LVB_DEM_H

#include <stdint.h>

#include "lvb.h"

#ifdef __cplusplus
extern "C" {
#endif

#define DEM_WALL_NONE     0
#define DEM_WALL_BOX      1
#define DEM_WALL_DRUM     2
#define DEM_WALL_SPECULAR 3

typedef struct {
    float kn;             /* normal stiffness [N/m] */
    float restitution;    /* e in (0, 1] */
    float rho;            /* density [kg/m^3] */
    float g[3];           /* gravity [m/s^2] */
    int32_t wall_kind;    /* DEM_WALL_* */
    int32_t clamp_tensile;/* 1: a negative (attractive) normal force is set to 0 */
    float drum_cx, drum_cz, drum_R, drum_omega;
    int32_t contacts_on;  /* 0: particles do not interact (ballistic runs) */
    int32_t pad;
    /* tangential law with contact history (LSD with static friction); on
     * when mu > 0, between particles only (walls stay frictionless): */
    float mu;             /* Coulomb coefficient: |F_t| <= mu max(F_n, 0) */
    float kt_ratio;       /* tangential stiffness k_t = kt_ratio k_n */
    float gt_ratio;       /* tangential damping gamma_t = gt_ratio gamma_n */
    int32_t pad2;
} dem_params;

typedef struct dem_ctx dem_ctx;

/* Phases of one step, for callers that time them separately. */
#define DEM_PHASE_INTEGRATE 0   /* x', v* */
#define DEM_PHASE_BROAD     1   /* lvb_step at x' (check + partial rebuild) */
#define DEM_PHASE_FORCES    2   /* narrow phase on the list, forces, a', v' */

/*
 * dem_init -- copy the initial state into library-owned device memory, build
 * the broad phase (lvb_init) at x0 and evaluate a0 = F(x0, v0)/m + g.
 *   pos_r, vel : device float4 (x, y, z, r) and (vx, vy, vz, -), n records.
 *   prm        : physics; dt > 0 the time step [s].
 *   box, skin, trigger, cell_factor : as lvb_init.
 * Synchronises.  Errors: EINVAL, ENOMEM, ENAN, EDEVICE.
 */
int dem_init(dem_ctx **out, int64_t n, const float *pos_r, const float *vel,
             const dem_params *prm, float dt, const lvb_box *box,
             const lvb_skin_policy *skin, int32_t trigger, float cell_factor,
             void *stream);

/*
 * dem_batch_init -- as dem_init over n_scenes independent scenes advancing
 * together (lvb_batch_init): scene s is particles [offsets[s],
 * offsets[s+1]) with its walls at boxes[s]; the physics (prm, dt) is shared.
 * offsets and boxes are host arrays.
 */
int dem_batch_init(dem_ctx **out, int32_t n_scenes, const int64_t *offsets,
                   const float *pos_r, const float *vel, const dem_params *prm, float dt,
                   const lvb_box *boxes, const lvb_skin_policy *skin, int32_t trigger,
                   float cell_factor, void *stream);

/* Steps captured in one CUDA graph by dem_advance. */
#define DEM_GRAPH_STEPS 100

/* dem_advance -- enqueue `steps` full steps (no synchronisation).  Chunks of
 * DEM_GRAPH_STEPS steps replay one CUDA graph, built node by node on first
 * use (and again after a store grew); the remainder runs as direct
 * launches.  Between chunks the host grows a store that asked to grow. */
int dem_advance(dem_ctx *ctx, int64_t steps);

/* dem_phase -- enqueue one phase (DEM_PHASE_*) of a step; a step is the
 * three phases in order. */
int dem_phase(dem_ctx *ctx, int32_t phase);

/* dem_get_rot_state -- copy out w, al (angular acceleration) and w*
 * (float4 records, w = 1/I in the first; any pointer may be NULL); all zero
 * without friction.  Synchronises. */
int dem_get_rot_state(dem_ctx *ctx, float *omega, float *alpha, float *omega_star);

/* dem_get_state -- copy out x (pos_r, with radii), v, a and v* (float4
 * records; the w of v and of v* holds 1 / m; any pointer may be NULL).
 * Synchronises. */
int dem_get_state(dem_ctx *ctx, float *pos_r, float *vel, float *acc, float *vstar);

/*
 * dem_get_contact_forces -- the contacts of the current state and the
 * normal force of each, as the forces phase evaluates them (the narrow
 * phase of Eq. delta on the list, the linear spring-dashpot law above):
 * every pair i < j of the list with delta_ij > 0 at the current positions
 * (x' of the last step), in no particular order, with
 *   force3 : the force on i, (k_n delta - gamma v_n) n_ij (3 floats a pair;
 *            the force on j is its negation),
 *   delta  : the overlap (compensated binary32).
 * ci, cj, force3, delta: host or device, cap entries (force3: 3 cap
 * floats); *n_contacts: the number of contacts (LVB_ECAPACITY if over cap,
 * the first cap written).  Allocates temporary device memory.
 * Synchronises.  Errors: EINVAL, ECAPACITY, ENOMEM, EDEVICE and the broad
 * phase's device errors.
 */
int dem_get_contact_forces(dem_ctx *ctx, int32_t *ci, int32_t *cj, float *force3, float *delta,
                           int64_t cap, int64_t *n_contacts);

/*
 * dem_get_contact_history -- as dem_get_contact_forces, with friction: the
 * force on i includes the tangential force, evaluated from the contact's
 * spring as the last step left it (F_t = -k_t xi - gamma_t v_t, which the
 * cap leaves equal to the capped force), and xi3 (3 floats a pair) gets
 * the spring xi of row i's record; xi3 may be NULL.  sides = 1: each pair
 * once, i < j; sides = 2: each pair from both rows, (i, j) and (j, i)
 * (their springs are exact negatives of each other).
 */
int dem_get_contact_history(dem_ctx *ctx, int32_t sides, int32_t *ci, int32_t *cj,
                            float *force3, float *delta, float *xi3, int64_t cap,
                            int64_t *n_contacts);

/* dem_set_state -- overwrite x, v, a (host or device float4 records; radii
 * in pos_r must equal the initial ones; the w of v is ignored, the driver
 * keeps 1 / m there).  The broad phase keeps its reference state, so the
 * next step's check sees the new positions. */
int dem_set_state(dem_ctx *ctx, const float *pos_r, const float *vel, const float *acc);

/* dem_lvb -- the broad-phase context the driver owns (valid until
 * dem_destroy), for lvb_get_* and lvb_stats. */
int dem_lvb(dem_ctx *ctx, lvb_ctx **out);

/* dem_device_state -- device pointers of the state arrays (float4 records),
 * owned by the context; for callers that read them in place. */
int dem_device_state(dem_ctx *ctx, float **pos_r, float **vel, float **acc, float **vstar);

/* dem_sync -- wait for the stream; returns the broad phase's sticky error. */
int dem_sync(dem_ctx *ctx);

int dem_destroy(dem_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LVB_DEM_H */
