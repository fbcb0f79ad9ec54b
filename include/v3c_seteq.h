/* Multiset-equality gadget (Sec. 4.5, Gadgets and Cost Model): the prover's
 * grand-product column of SetEq over compressed tuples.
 *
 *   Compress(t; beta) = sum_{k < T} t_k beta^k
 *   SetEq(X, Y):        prod_i (alpha - x_i) = prod_i (alpha - y_i)
 *   Z_0 = 1,  Z_{i+1} = Z_i (alpha - Compress(X_i)) / (alpha - Compress(Y_i))
 *
 * Z_L = 1 exactly when the two products agree.  For random alpha and beta,
 * that means the multisets of tuples agree (with high probability).  The GPU evaluates
 *   Z_i = [prod_{k<i} (alpha - x_k)] * [prod_{k>=i} (alpha - y_k)] * [prod_k (alpha - y_k)]^-1,
 * in tiles of 2048 elements: product scans inside a tile, the products of
 * the earlier tiles carried by a decoupled look-back, and one field
 * inversion per tile instead of one per element.  If some alpha - y_k is
 * zero, the inverse is taken as 0: the instance's whole column is then
 * written as zeros (Z_0 = 0 marks it), and its status is 1.
 *
 * All instances run in one scan launch (and one zeroing launch that only
 * touches degenerate instances).  Inputs are canonical, and
 * all pointers are device memory: X, Y [L][T] row-major, Z [L + 1].
 * Statuses: EINVAL (NULL pointer, T outside 1..32, L = 0 or L >= 2^40, or a
 * non-canonical alpha or beta), ENOMEM, ECUDA, ETIMEDOUT (a bounded wait of
 * the look-back gave up; reported when the call waits). */
#pragma once
#include "v3c.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    const uint64_t* x; /* [L][T] */
    const uint64_t* y; /* [L][T] */
    uint64_t* z;       /* [L + 1] */
    uint64_t L;
    uint32_t T;
    uint32_t pad;
    uint64_t alpha;
    uint64_t beta;
} v3c_seteq_desc;

/* Enqueues the grand-product columns of n instances on `stream`.  If
 * h_status is not NULL, the call waits and writes one status per instance
 * (0 = ok, 1 = alpha equals some compressed y); otherwise it returns
 * without waiting. */
v3c_status v3c_seteq(v3c_ctx* ctx, const v3c_seteq_desc* descs, uint32_t n, uint32_t* h_status, void* stream);

#ifdef __cplusplus
}
#endif
