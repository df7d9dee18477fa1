/*
 * lvb_clump.h -- narrow phase of multi-sphere clumps on the local Verlet
 * buffer list.
 *
 * The paper's broad phase works on bounding spheres and leaves the exact
 * shape to the narrow phase, naming multi-sphere clumps among the shapes it
 * serves (Sec. Background, the broad phase on bounding spheres and the
 * narrow phases that follow it).  Here a clump i is a rigid body of k_i
 * sub-spheres: the broad phase (lvb.h) runs on its bounding sphere
 * (x_i, R_i) as on any particle, and this call finds the contacts between
 * the sub-spheres of every clump pair of the list.
 *
 * Sub-sphere a of clump i, with body-frame offset b_a and radius r_a, sits
 * at x_a = x_i + R(q_i) b_a, q_i = (w, x, y, z) the clump's unit
 * quaternion and R(q) the rotation matrix
 *   [1 - 2(y y + z z)   2(x y - w z)       2(x z + w y)    ]
 *   [2(x y + w z)       1 - 2(x x + z z)   2(y z - w x)    ]
 *   [2(x z - w y)       2(y z + w x)       1 - 2(x x + y y)]
 * every product, sum and difference rounded to binary32 in the order
 * written (2 u rounded as 2 * u, s t as one product), and each component
 * of R b as ((R_k0 b_x + R_k1 b_y) + R_k2 b_z).  A contact is a pair of
 * sub-spheres a of i and b of j, i < j, with
 *   delta = (r_a + r_b) - sqrt(|x_a - x_b|^2) > 0
 * in the fixed binary32 formula of lvb.h (Eq. delta on sub-spheres).
 *
 * Every contact is found if each bounding radius covers its clump with a
 * margin for rounding: |b_a| + r_a <= R_i (1 - 2^-12) for every sub-sphere
 * (the call checks this, in binary64), and coordinates are at most 1e3
 * times the smallest bounding radius.
 */
#ifndef LVB_CLUMP_H
#define LVB_CLUMP_H

#include <stdint.h>

#include "lvb.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * lvb_clump_contacts -- the sub-sphere contacts of the clump pairs in the
 * context's list (the list built on the bounding spheres; the context's
 * radii are the bounding radii R_i).
 *   pos_r   : device, n float4 (x, y, z, R) -- the clumps' present positions
 *             and bounding radii (R as at lvb_init).
 *   quat    : device, n float4 (w, x, y, z) unit quaternions (|q| within
 *             2^-20 of 1).
 *   sub_off : device, n + 1 int32: clump i's sub-spheres are
 *             sub[sub_off[i] .. sub_off[i + 1]), at most 64 of them.
 *   sub     : device, float4 (b_x, b_y, b_z, r) per sub-sphere, body frame.
 *   ci, ca, cj, cb, delta : host or device out, cap entries each: contact k
 *             is sub-sphere ca[k] (its index within clump ci[k]) against
 *             sub-sphere cb[k] of clump cj[k], ci[k] < cj[k], overlap
 *             delta[k]; in no particular order.
 *   n_contacts : out, the number of contacts (LVB_ECAPACITY if over cap,
 *             the first cap written).
 * Outputs in device memory are written in place (no allocation); if any
 * output is in host memory, all five go through temporary device arrays
 * of cap entries.  Synchronises.  Errors: EINVAL (NULL or misaligned
 * pointers, a sub-sphere outside its bound's margin, a quaternion off unit
 * length, a negative first offset, offsets not increasing or more than 64
 * sub-spheres; nothing written), ECAPACITY, ENOMEM, EDEVICE, and the
 * context's device errors.
 */
int lvb_clump_contacts(lvb_ctx *ctx, const float *pos_r, const float *quat,
                       const int32_t *sub_off, const float *sub, int32_t *ci, int32_t *ca,
                       int32_t *cj, int32_t *cb, float *delta, int64_t cap,
                       int64_t *n_contacts);

#ifdef __cplusplus
}
#endif

#endif /* LVB_CLUMP_H */
