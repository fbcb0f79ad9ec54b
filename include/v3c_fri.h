/* FRI commit phase and batched openings on resident commitments.
 *
 * The paper's prover is Plonky2 with its default field, FRI parameters and
 * recursion layout (Sec. 5, evaluation environment).  It prints no FRI
 * formula; the operations below are the textbook FRI commit phase
 * (Ben-Sasson, Bentov, Horesh, Riabzev, ICALP 2018) run on the codewords
 * that v3c_commit leaves resident in HBM.
 *
 * Domain.  A committed LDE of N = 2^log_N rows has row t on the point
 * x_t = 7 * w_N^bitrev_{log N}(t).  The codeword of every FRI layer keeps
 * that bit-reversed order: layer k has N_k = 2^log_size[k] values on the
 * coset s_k * <w_{N_k}>, s_0 = 7, s_{k+1} = s_k^(2^a_k).  Positions 2u and
 * 2u+1 hold f(x) and f(-x), so every fold reads contiguous values.
 *
 * Combine.  f_0[t] = sum_i alpha^i M_t[i].  The M_t are the rows of the
 * listed commitments, concatenated in order (commitment 0's columns first),
 * so the exponent i runs on from one commitment to the next.  All listed
 * commitments must have the same row count.  The combination is plain; no
 * out-of-domain (DEEP) quotient is applied.
 *
 * Fold.  Round k folds 2^a_k values into one.  Write
 * f = sum_{i < 2^a} X^i f_i(X^(2^a)); then f_{k+1} = sum_i beta_k^i f_i, on
 * the squared coset.  The arity of round k is
 * a_k = min(arity_bits, log_size[k] - final_log), and rounds continue while
 * log_size[k] > final_log.
 *
 * Layer trees.  For k < R (R = the number of rounds), layer k is committed
 * as a Merkle tree of L_k = N_k / 2^a_k leaves.  Leaf w is the coset
 * f_k[w 2^a_k .. (w+1) 2^a_k), hashed like an LDE row of its 2^a_k values
 * (ext_degree words each): the Poseidon sponge, or zero padding when the
 * leaf has at most 4 words.  The cap height is
 * min(cap_height, log2 L_k).  The last layer f_R is not hashed; it is
 * returned as the coefficients of its polynomial (v3c_fri_final).
 *
 * Extension.  Plonky2's default FRI draws its challenges from a degree-2
 * extension.  With ext_degree = 2, alpha and the beta_k are elements
 * (re, im) = re + im u of F_p[u] / (u^2 - 7).  7 generates F_p^*, so u^2 - 7
 * is irreducible.  The combination, every layer and the final coefficients
 * are then pairs of words, (re, im) per value, and a leaf holds 2 * 2^a_k
 * words.  The LDE columns and the domain stay in F_p.  With ext_degree = 1,
 * everything is in F_p and a value is one word.
 *
 * Challenges.  alpha and the beta_k are inputs, ext_degree words each.  A
 * caller that derives beta_k from layer k's cap (Fiat-Shamir) passes no
 * betas to v3c_fri_begin,
 * reads cap 0, then calls v3c_fri_fold with one beta at a time.  A caller
 * that knows all betas passes them at once; the layer trees are then hashed
 * in one batched launch.
 *
 * All values are canonical Goldilocks elements (< p).  The calls enqueue
 * on `stream` (a cudaStream_t, NULL = legacy default stream) after the listed
 * commitments are complete.  The calls that return host data wait for the
 * work they read.  Statuses: EINVAL (bad argument, or a call out of order),
 * ENOTFOUND (unknown id), ENOMEM (HBM budget or allocation), ECUDA,
 * ETIMEDOUT (a bounded wait of the combination's copy pipeline gave up;
 * returned by the first call that reads a result of that FRI state back). */
#pragma once
#include "v3c.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef uint64_t v3c_fri_id;

typedef struct {
    uint32_t arity_bits; /* 1..4 */
    uint32_t final_log;  /* 0..10, below log_N */
    uint32_t cap_height; /* per-layer cap height, clamped to the layer's leaf count */
    uint32_t ext_degree; /* 1 (or 0): values in F_p; 2: in F_p[u]/(u^2 - 7) */
} v3c_fri_cfg;

#define V3C_FRI_MAX_ROUNDS 25
typedef struct {
    uint32_t rounds;      /* R */
    uint32_t rounds_done; /* folds applied so far (layers 0..rounds_done exist) */
    uint32_t log_N;       /* log_size[0] */
    uint32_t n_columns;   /* columns combined into f_0 */
    uint32_t arity_bits[V3C_FRI_MAX_ROUNDS];   /* a_k, k < R */
    uint32_t log_size[V3C_FRI_MAX_ROUNDS + 1]; /* log2 N_k, k <= R */
    uint32_t cap_height[V3C_FRI_MAX_ROUNDS];   /* of layer k's tree, k < R */
    uint64_t query_words; /* words per query written by v3c_fri_query */
    uint64_t bytes;       /* device bytes held by the state */
    uint32_t ext_degree;  /* 1 or 2: words per layer value */
    uint32_t pad;
} v3c_fri_info_t;

/* Starts the commit phase over n_ids resident commitments: allocates every
 * layer, builds f_0 and commits layer 0.  Then it applies the first n_betas
 * folds (n_betas <= R), as v3c_fri_fold does.  alpha points to ext_degree
 * words; h_betas to n_betas * ext_degree words.  The state counts against the
 * context's HBM budget until v3c_fri_release. */
v3c_status v3c_fri_begin(v3c_ctx* ctx, const v3c_commit_id* ids, uint32_t n_ids, const uint64_t* alpha,
                         const v3c_fri_cfg* cfg, const uint64_t* h_betas, uint32_t n_betas, v3c_fri_id* out,
                         void* stream);

/* Applies the next n_betas rounds: f_{k+1} = fold(f_k, beta_k), with
 * h_betas holding n_betas * ext_degree words.  Each new layer below R is
 * then committed.  When the last round is applied, the
 * final polynomial's coefficients are computed.  n_betas must not exceed the
 * rounds left. */
v3c_status v3c_fri_fold(v3c_ctx* ctx, v3c_fri_id fri, const uint64_t* h_betas, uint32_t n_betas, void* stream);

/* Round schedule and sizes of the state (host only, no wait). */
v3c_status v3c_fri_info(v3c_ctx* ctx, v3c_fri_id fri, v3c_fri_info_t* out);

/* Cap of layer k's tree: 2^cap_height[k] digests of 4 words.  The layer must
 * exist (k <= rounds_done, k < R). */
v3c_status v3c_fri_cap(v3c_ctx* ctx, v3c_fri_id fri, uint32_t layer, uint64_t* h_cap);

/* Coefficients of the last layer's polynomial: 2^log_size[R] values of
 * ext_degree words (re, im for degree 2), lowest degree first.  They are the
 * c_i with f_R(x_t) = sum_i c_i x_t^i on the layer's coset.  All rounds must be done.  For an honest prover, the
 * coefficients at and above deg / 2^(log_N - log_size[R]) are zero. */
v3c_status v3c_fri_final(v3c_ctx* ctx, v3c_fri_id fri, uint64_t* h_coeffs);

/* Batched query openings (all rounds done).  For each query position
 * t_0 = h_idx[q] < N the call writes query_words words at
 * h_out + q * query_words.  For each layer k < R, in order, they are:
 *   the 2^a_k values of leaf w_k = t_k >> a_k, ext_degree words each, where
 *   t_k = t_0 >> (a_0 + ... + a_{k-1});
 *   its Merkle path, the siblings level_j[(w_k >> j) ^ 1] for
 *   j = 0 .. log2 L_k - cap_height[k] - 1, 4 words each.
 * The initial rows at t_0 come from v3c_open_batch on the commitments. */
v3c_status v3c_fri_query(v3c_ctx* ctx, v3c_fri_id fri, const uint64_t* h_idx, uint32_t nq, uint64_t* h_out);

/* Frees the state (stream-ordered after its last work). */
v3c_status v3c_fri_release(v3c_ctx* ctx, v3c_fri_id fri);

/* Batched Merkle openings of a resident commitment (MerkleOpen, Sec. 4.4).
 * For each leaf index t = h_leaves[q] < N it writes the committed row
 * (c words, at h_rows + q * c) and the authentication path
 * (log_N - h digests of 4 words, at h_paths + q * 4 * (log_N - h)).  The
 * path holds the siblings level_k[(t >> k) ^ 1], k = 0 .. log_N - h - 1.
 * Either output may be NULL.  One gather launch and one copy back, whatever
 * nq is. */
v3c_status v3c_open_batch(v3c_ctx* ctx, v3c_commit_id id, const uint64_t* h_leaves, uint32_t nq, uint64_t* h_rows,
                          uint64_t* h_paths);

#ifdef __cplusplus
}
#endif
