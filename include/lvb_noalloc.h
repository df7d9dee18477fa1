/*
 * lvb_noalloc.h -- a neighbour-list build that allocates no memory.
 *
 * The paper has no counterpart to this entry point: its method keeps a list
 * inside a running simulation (lvb.h).  This call serves callers that may
 * not allocate -- code running under another framework's allocator or a
 * fixed memory budget, plug-ins that must not change the process's device
 * footprint, loops where an allocation may neither fail nor stall.  It
 * builds, once, the list a context would hold for the given reference
 * state, with working memory in a fixed device array inside the library.
 */
#ifndef LVB_NOALLOC_H
#define LVB_NOALLOC_H

#include <stdint.h>

#include "lvb.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest n that lvb_pairs_noalloc takes.  Its working memory (cell counts
 * and offsets, and the reference records sorted by cell: about 1.6 MB) is a
 * file-scope device array of the library, sized for this many particles and
 * for at most 32768 cells; larger boxes get coarser cells, never more
 * memory. */
#define LVB_NOALLOC_MAX_N 65536

/*
 * lvb_pairs_noalloc -- every pair i < j with
 *   |xref_i - xref_j|^2 <= (R_NL,i + R_NL,j)^2,   R_NL = r + skin
 * on the reference positions, each sum, difference and product rounded to
 * binary32 in the order lvb.h gives (no fused multiply-add), i.e. the pair
 * set that lvb_get_pairs_ij returns for a context holding the same
 * reference state, in no particular order.
 *
 *   n       : number of particles, 1 <= n <= LVB_NOALLOC_MAX_N.
 *   pos4    : device, n float4 records (x, y, z, r); only r is read.
 *             16-byte aligned.  r > 0, finite.
 *   ref4    : device, n float4 records (xref, yref, zref, skin), e.g. from
 *             lvb_get_ref.  16-byte aligned.  Finite, skin >= 0.
 *   box     : host; the cell grid spans it, positions outside fall in the
 *             border cells (correct, only slower).  hi > lo on every axis.
 *   pi, pj  : device, cap int32 each (may be NULL if cap == 0); receive the
 *             first min(count, cap) pairs.  Owned by the caller.
 *   cap     : capacity of pi and pj, >= 0.
 *   n_pairs : host out, the number of pairs (also when it exceeds cap).
 *   stream  : CUDA stream (NULL = legacy default stream) on the current
 *             device; the call synchronises it twice (it reads the largest
 *             R_NL to size the cells, then the pair count).
 *
 * Returns LVB_OK; LVB_ECAPACITY when the count exceeds cap (pi, pj hold
 * the first cap pairs found, *n_pairs the full count); LVB_ELIMIT when
 * n > LVB_NOALLOC_MAX_N (nothing is launched); LVB_EINVAL for NULL or
 * misaligned pointers, n < 1, cap < 0, a bad box, r <= 0 or skin < 0;
 * LVB_ENAN for a non-finite input; LVB_EDEVICE when a CUDA call fails.
 * An error of the caller's own earlier CUDA work that the caller has not
 * yet read (cudaGetLastError) is left in place: this call reads the status
 * of each of its own launches and copies directly.
 *
 * No memory is allocated -- no cudaMalloc, cudaFree or allocating library
 * call, on the device or the host.  The first call on a device does a
 * one-time set-up: it looks up the device address of the working array
 * (cudaGetSymbolAddress with that device current, which may also load
 * the library's module there).  The call cannot be captured into a CUDA
 * graph (it synchronises its stream and reads results to the host): on a
 * stream that is capturing, or whose capture status cannot be read, it
 * returns LVB_EINVAL before any launch.  Nothing needs to start at zero: each call clears its counters
 * and cell counts on the stream before use.  All calls on one device share
 * the one working array, so calls that overlap in time on that device --
 * from two host threads, or on two streams -- race on it and give wrong
 * lists; serialise them.
 */
int lvb_pairs_noalloc(int64_t n, const float *pos4, const float *ref4, const lvb_box *box,
                      int32_t *pi, int32_t *pj, int64_t cap, int64_t *n_pairs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LVB_NOALLOC_H */
