/* Snapshot commitment of a fixed-shape IVF-PQ index (Sec. 4.3, Snapshot
 * Commitments), built on the GPU with the same Poseidon sponge and Merkle
 * compression as the polynomial commitments.
 *
 * Inputs (all canonical field elements, row-major):
 *   records   [nlist * n][2 + M]  slot (i, j) at row i * n + j, holding
 *             (f_{i,j}, item_{i,j}, v_{i,j}^(0), ..., v_{i,j}^(M-1));
 *   centroids [nlist][D]          mu_i, fixed-point coordinates;
 *   codebooks [M][K][d]           C_{m,k} in F^d, flattened in that order.
 * nlist = 2^log_nlist and n = 2^log_n (full balanced trees, Sec. 4.3).
 *
 * Outputs:
 *   hash_{i,j} = Hash(i, j, f_{i,j}, item_{i,j}, v_{i,j}^(0..M-1))
 *   root_i     = MerkleTree(hash_{i,0}, ..., hash_{i,n-1})
 *   hash_i     = Hash(i, mu_i, root_i)
 *   root_mk    = MerkleTree(hash_0, ..., hash_{nlist-1})
 *   root_cb    = Hash(C_{0,0}, ..., C_{M-1,K-1})
 * Hash is the Poseidon-w12 sponge (rate 8, overwrite mode, 4-word digest;
 * an input of at most 4 words is its own zero-padded digest).  MerkleTree
 * takes digests as leaves, node = Perm(L || R || 0^4)[0..4), up to one root.
 *
 * The snapshot object keeps the list roots, the centroid digests and the
 * top-level tree resident.  These are what the snapshot-binding circuit
 * takes as witness: every root_i, and the top-level path pi_i of each probed
 * list.  The slot-level trees are scratch, freed after the build.
 * Statuses: EINVAL, ENOTFOUND, ENOMEM (HBM budget or allocation), ECUDA. */
#pragma once
#include "v3c.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef uint64_t v3c_snapshot_id;

typedef struct {
    const uint64_t* records;   /* [nlist * n][2 + M] */
    const uint64_t* centroids; /* [nlist][D] */
    const uint64_t* codebooks; /* [M][K][d] */
    int on_device;             /* V3C_INPUT_DEVICE: device pointers; otherwise host memory, copied */
    uint32_t log_nlist;        /* <= 20 */
    uint32_t log_n;            /* log_nlist + log_n <= 26 */
    uint32_t M;                /* PQ sub-quantizers, 1..64 */
    uint32_t D;                /* centroid dimension, 1..65536 */
    uint32_t K;                /* codewords per sub-quantizer, >= 1 */
    uint32_t d;                /* codeword dimension, >= 1; M * K * d < 2^31 */
} v3c_snapshot_desc;

/* Builds the commitment on `stream` (a cudaStream_t) and returns a resident
 * snapshot object.  The codebook digest, a single sequential sponge, runs on
 * a second stream alongside the tree levels and is joined back before the
 * call's work on `stream` completes.  The context keeps a device copy of the
 * last committed codebooks and their digest: a commit whose codebooks are
 * equal word for word (compared on the device) reuses the digest, so
 * successive snapshot versions with unchanged codebooks skip the sponge.
 * Host inputs are copied before the call returns. */
v3c_status v3c_snapshot_commit(v3c_ctx* ctx, const v3c_snapshot_desc* desc, v3c_snapshot_id* out, void* stream);

/* root_mk and root_cb (4 words each; either may be NULL).  Waits for the build. */
v3c_status v3c_snapshot_roots(v3c_ctx* ctx, v3c_snapshot_id id, uint64_t* h_root_mk, uint64_t* h_root_cb);

/* The list roots [nlist][4] (witness of the snapshot-binding circuit). */
v3c_status v3c_snapshot_list_roots(v3c_ctx* ctx, v3c_snapshot_id id, uint64_t* h_roots);

/* Top-level Merkle paths pi_i of the lists h_lists[q] < nlist: log_nlist
 * sibling digests each (the siblings hash_.[(i >> k) ^ 1], k = 0 ..
 * log_nlist - 1, with level k of the top-level tree), written at
 * h_paths + q * 4 * log_nlist.  One gather launch and one copy back. */
v3c_status v3c_snapshot_open_lists(v3c_ctx* ctx, v3c_snapshot_id id, const uint32_t* h_lists, uint32_t nq,
                                   uint64_t* h_paths);

/* Frees the object (stream-ordered after its build). */
v3c_status v3c_snapshot_release(v3c_ctx* ctx, v3c_snapshot_id id);

#ifdef __cplusplus
}
#endif
