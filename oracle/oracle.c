/*
 * CPU oracle for the V3DB polynomial commitment (coset LDE + Poseidon-w12
 * Merkle tree).  TEST INFRASTRUCTURE ONLY: nothing on the product path may
 * call, link or load this file.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it.
 *
 * It is written to be slow and obviously correct:
 *   - field arithmetic uses unsigned __int128 and the `%` operator,
 *   - the NTT is a recursive radix-2 decimation-in-time taken from the DFT
 *     definition, natural order in and out,
 *   - the LDE zero-pads to the full N = n * 2^r domain and runs one size-N
 *     NTT (no coset splitting),
 *   - Poseidon is the textbook round loop (ARC -> S-box -> dense MDS).
 * The only concession to speed is a parallel-for over independent columns,
 * leaves or tree nodes.  It shares no code, header or constant table with
 * the CUDA library: the Poseidon constants are re-derived here from the
 * seeded generator's definition.
 *
 * Paper context (V3DB, arXiv 2603.03065): the prover is "based on Plonky2"
 * (abstract) with the default Plonky2 field and FRI setup (Sec. 5,
 * evaluation environment); proving cost lives in FFT-based polynomial
 * operations over a padded power-of-two domain G_B = 2^ceil(log2 G)
 * (Sec. 2.1, "binning effect"); the hash is Poseidon (Sec. 4.3) and
 * commitments are balanced Merkle trees whose openings follow the bits of
 * the leaf index (Sec. 4.3, Sec. 4.4 MerkleOpen).  The paper fixes none of
 * the numeric parameters; the readings used here are:
 *   field  p = 2^64 - 2^32 + 1, multiplicative generator 7;
 *   LDE    a = iNTT_n(col), b_i = a_i * 7^i, zero-pad to N, E = NTT_N(b),
 *          committed row t holds E[bitrev_{log N}(t)];
 *   hash   Poseidon width 12, rate 8, capacity 4, x^7, rounds 4 full +
 *          22 partial + 4 full, each round ARC -> S-box -> MDS, partial
 *          S-box on lane 0 only; constants from SplitMix64 (seed
 *          "V3DBPOS1"), MDS = first small-entry circulant with every square
 *          minor nonzero;
 *   sponge overwrite mode, no padding, 4-element digest, inputs of length
 *          <= 4 are zero-padded instead of hashed;
 *   tree   node = Perm(L || R || 0^4)[0..4), cut at a cap of 2^h digests.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

#define ORC_P 0xFFFFFFFF00000001ULL

/* ------------------------------------------------------------------ */
/* Field F_p with p = 2^64 - 2^32 + 1 (Goldilocks), plain % reduction.  */
/* ------------------------------------------------------------------ */

u64 orc_add(u64 a, u64 b) { return (u64)(((u128)a + b) % ORC_P); }
u64 orc_sub(u64 a, u64 b) { return (u64)(((u128)a + ORC_P - b) % ORC_P); }
u64 orc_mul(u64 a, u64 b) { return (u64)(((u128)a * b) % ORC_P); }

u64 orc_pow(u64 a, u64 e)
{
    u64 r = 1, x = a % ORC_P;
    while (e) {
        if (e & 1) r = orc_mul(r, x);
        x = orc_mul(x, x);
        e >>= 1;
    }
    return r;
}

/* Fermat inverse a^(p-2); inv(0) returns 0. */
u64 orc_inv(u64 a) { return orc_pow(a, ORC_P - 2); }

/* omega_m = 7^((p-1)/m): a primitive m-th root of unity for m = 2^log_m,
 * log_m <= 32 (p - 1 = 2^32 * 3 * 5 * 17 * 257 * 65537, 7 generates F_p^*). */
u64 orc_root_of_unity(uint32_t log_m)
{
    if (log_m > 32) return 0;
    return orc_pow(7, (ORC_P - 1) >> log_m);
}

static uint32_t bitrev(uint64_t x, uint32_t bits)
{
    uint64_t r = 0;
    for (uint32_t i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
    return (uint32_t)r;
}
uint32_t orc_bitrev(uint64_t x, uint32_t bits) { return bitrev(x, bits); }

/* ------------------------------------------------------------------ */
/* Simple parallel-for over [0, n) with pthreads.                       */
/* ------------------------------------------------------------------ */

typedef void (*orc_body)(void* ctx, size_t i);
typedef struct {
    orc_body fn;
    void* ctx;
    size_t n;
    size_t next;
    pthread_mutex_t mu;
} pf_state;

static void* pf_worker(void* arg)
{
    pf_state* st = (pf_state*)arg;
    for (;;) {
        size_t i;
        pthread_mutex_lock(&st->mu);
        i = st->next++;
        pthread_mutex_unlock(&st->mu);
        if (i >= st->n) break;
        st->fn(st->ctx, i);
    }
    return NULL;
}

static void parallel_for(size_t n, int threads, orc_body fn, void* ctx)
{
    if (threads <= 1 || n <= 1) {
        for (size_t i = 0; i < n; i++) fn(ctx, i);
        return;
    }
    if ((size_t)threads > n) threads = (int)n;
    pf_state st;
    st.fn = fn;
    st.ctx = ctx;
    st.n = n;
    st.next = 0;
    pthread_mutex_init(&st.mu, NULL);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    int started = 0;
    for (int t = 0; t < threads; t++) {
        if (pthread_create(&th[t], NULL, pf_worker, &st) == 0) started++;
        else break;
    }
    if (started == 0) pf_worker(&st);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&st.mu);
}

/* ------------------------------------------------------------------ */
/* NTT: X_j = sum_i x_i w^{ij}, straight from the definition, by the    */
/* even/odd split X_j = E_j + w^j O_j, X_{j+m/2} = E_j - w^j O_j.        */
/* (Sec. 2.1: the prover's cost is FFT-based polynomial arithmetic on a */
/* power-of-two domain.)                                                */
/* ------------------------------------------------------------------ */

static void ntt_rec(const u64* x, size_t stride, size_t m, u64 w, u64* out)
{
    if (m == 1) {
        out[0] = x[0];
        return;
    }
    size_t h = m / 2;
    u64 w2 = orc_mul(w, w);
    ntt_rec(x, 2 * stride, h, w2, out);          /* E: even-indexed inputs */
    ntt_rec(x + stride, 2 * stride, h, w2, out + h); /* O: odd-indexed inputs */
    u64 wj = 1;
    for (size_t j = 0; j < h; j++) {
        u64 e = out[j];
        u64 o = orc_mul(out[h + j], wj);
        out[j] = orc_add(e, o);
        out[h + j] = orc_sub(e, o);
        wj = orc_mul(wj, w);
    }
}

/* In-place NTT of size 2^log_m (natural order in and out).  inverse != 0
 * computes iNTT_m(X)_i = m^{-1} sum_j X_j w^{-ij}.  Returns 0 on success. */
int orc_ntt(u64* x, uint32_t log_m, int inverse)
{
    if (log_m > 32) return -1;
    size_t m = (size_t)1 << log_m;
    u64* out = (u64*)malloc(m * sizeof(u64));
    if (!out) return -1;
    u64 w = orc_root_of_unity(log_m);
    if (inverse) w = orc_inv(w);
    ntt_rec(x, 1, m, w, out);
    if (inverse) {
        u64 minv = orc_inv((u64)m % ORC_P);
        for (size_t i = 0; i < m; i++) out[i] = orc_mul(out[i], minv);
    }
    memcpy(x, out, m * sizeof(u64));
    free(out);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Coset low-degree extension of one column (definition as read for    */
/* the Plonky2-style commitment the paper's prover uses, Sec. 5):        */
/*   a = iNTT_n(col); b_i = a_i 7^i (i < n), 0 (n <= i < N); E = NTT_N(b) */
/* so E_j = P(7 w_N^j) with P(x) = sum a_i x^i; row t holds E_bitrev(t). */
/* ------------------------------------------------------------------ */

typedef struct {
    const u64* cols;
    uint32_t c, log_n, r, ld;
    u64* lde;
    int status;
} lde_ctx;

static void lde_column(void* vctx, size_t col)
{
    lde_ctx* L = (lde_ctx*)vctx;
    size_t n = (size_t)1 << L->log_n;
    uint32_t log_N = L->log_n + L->r;
    size_t N = (size_t)1 << log_N;
    u64* b = (u64*)calloc(N, sizeof(u64));
    if (!b) {
        L->status = -1;
        return;
    }
    memcpy(b, L->cols + col * n, n * sizeof(u64));
    orc_ntt(b, L->log_n, 1);                 /* coefficients a_i */
    u64 gi = 1;
    for (size_t i = 0; i < n; i++) {         /* coset shift by the generator */
        b[i] = orc_mul(b[i], gi);
        gi = orc_mul(gi, 7);
    }
    orc_ntt(b, log_N, 0);                    /* evaluations on 7 * <w_N> */
    for (size_t t = 0; t < N; t++)
        L->lde[t * L->ld + col] = b[bitrev(t, log_N)];
    free(b);
}

/* cols: column-major [c][n]; lde: row-major [N][ld], bit-reversed rows,
 * columns c..ld-1 zero.  Returns 0 on success. */
int orc_lde(const u64* cols, uint32_t c, uint32_t log_n, uint32_t r, u64* lde, uint32_t ld,
            int threads)
{
    if (ld < c || log_n + r > 30) return -1;
    size_t N = (size_t)1 << (log_n + r);
    for (size_t t = 0; t < N; t++)
        for (uint32_t j = c; j < ld; j++) lde[t * ld + j] = 0;
    lde_ctx L = {cols, c, log_n, r, ld, lde, 0};
    parallel_for(c, threads, lde_column, &L);
    return L.status;
}

/* Coefficients of every column: coeffs[j][i] = a_i of column j. */
typedef struct {
    const u64* cols;
    u64* coeffs;
    uint32_t log_n;
} coef_ctx;
static void coef_column(void* vctx, size_t col)
{
    coef_ctx* C = (coef_ctx*)vctx;
    size_t n = (size_t)1 << C->log_n;
    memcpy(C->coeffs + col * n, C->cols + col * n, n * sizeof(u64));
    orc_ntt(C->coeffs + col * n, C->log_n, 1);
}
int orc_coeffs(const u64* cols, uint32_t c, uint32_t log_n, u64* coeffs, int threads)
{
    coef_ctx C = {cols, coeffs, log_n};
    parallel_for(c, threads, coef_column, &C);
    return 0;
}

/* LDE rows by direct evaluation: for each requested committed row t, the
 * point is x = 7 * w_N^{bitrev(t)} and row[j] = P_j(x) by Horner's rule on
 * the coefficients from orc_coeffs.  Used for sampled checks at sizes where
 * the full NTT-based oracle would take too long. */
typedef struct {
    const u64* coeffs;
    uint32_t c, log_n, r;
    const uint64_t* rows;
    u64* out;
} eval_ctx;
static void eval_row(void* vctx, size_t k)
{
    eval_ctx* E = (eval_ctx*)vctx;
    size_t n = (size_t)1 << E->log_n;
    uint32_t log_N = E->log_n + E->r;
    u64 x = orc_mul(7, orc_pow(orc_root_of_unity(log_N), bitrev(E->rows[k], log_N)));
    for (uint32_t j = 0; j < E->c; j++) {
        const u64* a = E->coeffs + (size_t)j * n;
        u64 acc = 0;
        for (size_t i = n; i-- > 0;) acc = orc_add(orc_mul(acc, x), a[i]);
        E->out[k * E->c + j] = acc;
    }
}
int orc_lde_rows(const u64* coeffs, uint32_t c, uint32_t log_n, uint32_t r, const uint64_t* rows,
                 uint32_t nrows, u64* out, int threads)
{
    eval_ctx E = {coeffs, c, log_n, r, rows, out};
    parallel_for(nrows, threads, eval_row, &E);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Poseidon-w12 constants from the seeded generator.                    */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the state advances by  */
/* the golden-ratio increment and each output is the state passed       */
/* through two xor-shift-multiply steps and a final xor-shift.          */
/* ------------------------------------------------------------------ */

static u64 splitmix64_next(u64* state)
{
    u64 z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
u64 orc_splitmix64_next(u64* state) { return splitmix64_next(state); }

#define ORC_W 12
#define ORC_ROUNDS 30
#define ORC_RF_HALF 4
/* Seed: the ASCII bytes "V3DBPOS1" read as a big-endian u64. */
#define ORC_SEED 0x56334442504F5331ULL

static u64 g_rc[ORC_ROUNDS][ORC_W];
static u64 g_mds[ORC_W][ORC_W];
static u64 g_mds_row[ORC_W];
static uint32_t g_mds_tries;
static int g_params_ready;
static pthread_once_t g_params_once = PTHREAD_ONCE_INIT;

/* Rank of a 12-bit mask among the masks with the same popcount. */
static int g_rank[1 << ORC_W];
static int g_count[ORC_W + 1];
static uint16_t g_masks[ORC_W + 1][924];

static void build_rank_tables(void)
{
    memset(g_count, 0, sizeof g_count);
    for (int m = 0; m < (1 << ORC_W); m++) {
        int k = __builtin_popcount((unsigned)m);
        g_rank[m] = g_count[k];
        g_masks[k][g_count[k]] = (uint16_t)m;
        g_count[k]++;
    }
}

/* Every square minor of the 12x12 matrix A is nonzero mod p (the MDS
 * condition).  Minors are computed by Laplace expansion along the smallest
 * row of each row set, memoising the minors of the previous size: the
 * minor on rows R and columns C (|R| = |C| = k) is
 *   sum over the idx-th column c of C of (-1)^idx A[min R][c] * minor(R \ min R, C \ c).
 * Returns 1 if all C(24,12) - 1 minors are nonzero, 0 if one vanishes,
 * -1 on allocation failure. */
int orc_mds_check(const u64* A /* row-major 12x12 */)
{
    static pthread_once_t once = PTHREAD_ONCE_INIT;
    pthread_once(&once, build_rank_tables);
    u64* prev = (u64*)malloc(sizeof(u64) * 924 * 924);
    u64* cur = (u64*)malloc(sizeof(u64) * 924 * 924);
    if (!prev || !cur) {
        free(prev);
        free(cur);
        return -1;
    }
    /* size 1 */
    for (int ri = 0; ri < g_count[1]; ri++)
        for (int ci = 0; ci < g_count[1]; ci++) {
            int r = __builtin_ctz(g_masks[1][ri]), c = __builtin_ctz(g_masks[1][ci]);
            u64 v = A[r * ORC_W + c] % ORC_P;
            if (v == 0) {
                free(prev);
                free(cur);
                return 0;
            }
            prev[ri * g_count[1] + ci] = v;
        }
    for (int k = 2; k <= ORC_W; k++) {
        int nk = g_count[k], nk1 = g_count[k - 1];
        for (int ri = 0; ri < nk; ri++) {
            int R = g_masks[k][ri];
            int r0 = __builtin_ctz((unsigned)R);
            int Rrest = g_rank[R & ~(1 << r0)];
            for (int ci = 0; ci < nk; ci++) {
                int C = g_masks[k][ci];
                u64 acc = 0;
                int idx = 0;
                for (int c = 0; c < ORC_W; c++) {
                    if (!(C & (1 << c))) continue;
                    u64 term = orc_mul(A[r0 * ORC_W + c] % ORC_P,
                                       prev[Rrest * nk1 + g_rank[C & ~(1 << c)]]);
                    acc = (idx & 1) ? orc_sub(acc, term) : orc_add(acc, term);
                    idx++;
                }
                if (acc == 0) {
                    free(prev);
                    free(cur);
                    return 0;
                }
                cur[ri * nk + ci] = acc;
            }
        }
        u64* t = prev;
        prev = cur;
        cur = t;
    }
    free(prev);
    free(cur);
    return 1;
}

/* Constant derivation:
 *   RC[rho][i], rho-major: successive SplitMix64 draws, each kept iff < p;
 *   MDS: candidate first rows of 12 entries, each entry (draw & 63) with 0
 *   redrawn; the circulant M[i][j] = m[(j - i) mod 12] of the first
 *   candidate that passes the minors check is the MDS. */
static void derive_params(void)
{
    u64 st = ORC_SEED;
    for (int rho = 0; rho < ORC_ROUNDS; rho++)
        for (int i = 0; i < ORC_W; i++) {
            u64 d;
            do d = splitmix64_next(&st);
            while (d >= ORC_P);
            g_rc[rho][i] = d;
        }
    for (uint32_t tries = 1; tries < 100000; tries++) {
        u64 row[ORC_W];
        for (int i = 0; i < ORC_W; i++) {
            u64 e;
            do e = splitmix64_next(&st) & 63;
            while (e == 0);
            row[i] = e;
        }
        u64 M[ORC_W * ORC_W];
        for (int i = 0; i < ORC_W; i++)
            for (int j = 0; j < ORC_W; j++) M[i * ORC_W + j] = row[(j - i + ORC_W) % ORC_W];
        if (orc_mds_check(M) == 1) {
            memcpy(g_mds_row, row, sizeof row);
            for (int i = 0; i < ORC_W; i++)
                for (int j = 0; j < ORC_W; j++) g_mds[i][j] = M[i * ORC_W + j];
            g_mds_tries = tries;
            g_params_ready = 1;
            return;
        }
    }
}

static int params(void)
{
    pthread_once(&g_params_once, derive_params);
    return g_params_ready;
}

/* Exports the derived constants: rc[360] round-major, mds[144] row-major,
 * returns the number of candidate rows drawn (0 if the search failed). */
uint32_t orc_poseidon_params(u64* rc, u64* mds)
{
    if (!params()) return 0;
    if (rc) memcpy(rc, g_rc, sizeof g_rc);
    if (mds) memcpy(mds, g_mds, sizeof g_mds);
    return g_mds_tries;
}

/* ------------------------------------------------------------------ */
/* Poseidon permutation (Poseidon paper, Grassi et al. USENIX Sec. 2021, */
/* HADES design; Sec. 4.3 names Poseidon as the hash): rounds 0-3 and   */
/* 26-29 full, 4-25 partial; each round ARC, S-box x^7, then MDS.       */
/* ------------------------------------------------------------------ */

static u64 sbox(u64 x)
{
    u64 x2 = orc_mul(x, x);
    u64 x3 = orc_mul(x2, x);
    u64 x4 = orc_mul(x2, x2);
    return orc_mul(x3, x4);
}

void orc_permute(u64* s /* [12], canonical */)
{
    params();
    for (int rho = 0; rho < ORC_ROUNDS; rho++) {
        for (int i = 0; i < ORC_W; i++) s[i] = orc_add(s[i], g_rc[rho][i]);
        int full = rho < ORC_RF_HALF || rho >= ORC_ROUNDS - ORC_RF_HALF;
        if (full)
            for (int i = 0; i < ORC_W; i++) s[i] = sbox(s[i]);
        else
            s[0] = sbox(s[0]);
        u64 t[ORC_W];
        for (int i = 0; i < ORC_W; i++) {
            u128 acc = 0; /* 12 * 63 * p < 2^74: no overflow */
            for (int j = 0; j < ORC_W; j++) acc += (u128)g_mds[i][j] * s[j];
            t[i] = (u64)(acc % ORC_P);
        }
        memcpy(s, t, sizeof t);
    }
}

/* Sponge hash, overwrite mode: state starts at zero; each chunk of up to
 * 8 inputs overwrites lanes 0..len-1 (other lanes kept) and is followed by
 * one permutation; the digest is lanes 0..3.  Inputs of length <= 4 are
 * returned zero-padded to 4 without hashing. */
void orc_hash(const u64* x, uint32_t len, u64* out /* [4] */)
{
    if (len <= 4) {
        for (uint32_t i = 0; i < 4; i++) out[i] = i < len ? x[i] : 0;
        return;
    }
    u64 s[ORC_W] = {0};
    for (uint32_t start = 0; start < len; start += 8) {
        uint32_t n = len - start < 8 ? len - start : 8;
        for (uint32_t i = 0; i < n; i++) s[i] = x[start + i];
        orc_permute(s);
    }
    memcpy(out, s, 4 * sizeof(u64));
}

/* Two-to-one compression C(L, R) = Perm(L || R || 0^4)[0..4). */
void orc_compress(const u64* l, const u64* r, u64* out)
{
    u64 s[ORC_W] = {0};
    memcpy(s, l, 4 * sizeof(u64));
    memcpy(s + 4, r, 4 * sizeof(u64));
    orc_permute(s);
    memcpy(out, s, 4 * sizeof(u64));
}

/* ------------------------------------------------------------------ */
/* Merkle tree over the rows (Sec. 4.3: balanced tree over a power-of-  */
/* two number of leaves; Sec. 4.4: the opening walks up by the bits of  */
/* the leaf index, left child = even index).                            */
/* tree: level-major, levels 0 .. logN-h-1 (level k has N >> k digests  */
/* of 4 elements); cap: the 2^h digests of level logN-h.                */
/* ------------------------------------------------------------------ */

typedef struct {
    const u64* rows;
    uint32_t ld, width;
    u64* leaves;
} leaf_ctx;
static void leaf_body(void* vctx, size_t t)
{
    leaf_ctx* L = (leaf_ctx*)vctx;
    orc_hash(L->rows + t * L->ld, L->width, L->leaves + 4 * t);
}

typedef struct {
    const u64* below;
    u64* above;
} level_ctx;
static void level_body(void* vctx, size_t u)
{
    level_ctx* L = (level_ctx*)vctx;
    orc_compress(L->below + 8 * u, L->below + 8 * u + 4, L->above + 4 * u);
}

/* Leaf digests of `nrows` rows (row-major, stride ld, width hashed). */
int orc_leaf_hashes(const u64* rows, uint32_t ld, uint32_t width, uint64_t nrows, u64* out,
                    int threads)
{
    if (!params()) return -1;
    leaf_ctx L = {rows, ld, width, out};
    parallel_for(nrows, threads, leaf_body, &L);
    return 0;
}

/* One tree level: above[u] = C(below[2u], below[2u+1]) for u < count. */
int orc_merkle_level(const u64* below, uint64_t count, u64* above, int threads)
{
    if (!params()) return -1;
    level_ctx L = {below, above};
    parallel_for(count, threads, level_body, &L);
    return 0;
}

int orc_merkle(const u64* rows, uint32_t ld, uint32_t width, uint32_t log_rows, uint32_t h,
               u64* tree, u64* cap, int threads)
{
    if (h > log_rows || !params()) return -1;
    size_t N = (size_t)1 << log_rows;
    u64* level = (u64*)malloc(N * 4 * sizeof(u64));
    if (!level) return -1;
    orc_leaf_hashes(rows, ld, width, N, level, threads);
    size_t off = 0, cnt = N;
    for (uint32_t k = 0; k < log_rows - h; k++) {
        memcpy(tree + off, level, cnt * 4 * sizeof(u64));
        off += cnt * 4;
        u64* next = (u64*)malloc((cnt / 2) * 4 * sizeof(u64));
        if (!next) {
            free(level);
            return -1;
        }
        orc_merkle_level(level, cnt / 2, next, threads);
        free(level);
        level = next;
        cnt /= 2;
    }
    memcpy(cap, level, cnt * 4 * sizeof(u64));
    free(level);
    return 0;
}

/* Authentication path of leaf t from a level-major tree: the sibling
 * level_k[(t >> k) ^ 1] for k = 0 .. logN-h-1. */
int orc_merkle_path(const u64* tree, uint32_t log_rows, uint32_t h, uint64_t t, u64* path)
{
    if (h > log_rows || t >> log_rows) return -1;
    size_t off = 0, cnt = (size_t)1 << log_rows;
    for (uint32_t k = 0; k < log_rows - h; k++) {
        size_t sib = (size_t)((t >> k) ^ 1);
        memcpy(path + 4 * k, tree + off + 4 * sib, 4 * sizeof(u64));
        off += cnt * 4;
        cnt /= 2;
    }
    return 0;
}

/* MerkleOpen (Sec. 4.4): hash the row, fold in the siblings by the bits
 * of t, compare with cap[t >> (logN - h)].  Returns 1 if it verifies. */
int orc_merkle_verify(const u64* row, uint32_t width, uint32_t log_rows, uint32_t h, uint64_t t,
                      const u64* path, const u64* cap)
{
    if (h > log_rows || t >> log_rows) return 0;
    u64 d[4], tmp[4];
    orc_hash(row, width, d);
    for (uint32_t k = 0; k < log_rows - h; k++) {
        if ((t >> k) & 1) orc_compress(path + 4 * k, d, tmp);
        else orc_compress(d, path + 4 * k, tmp);
        memcpy(d, tmp, sizeof d);
    }
    const u64* c = cap + 4 * (t >> (log_rows - h));
    return memcmp(d, c, sizeof d) == 0;
}

/* Whole commitment: LDE then Merkle tree. */
int orc_commit(const u64* cols, uint32_t c, uint32_t log_n, uint32_t r, uint32_t h, u64* lde,
               uint32_t ld, u64* tree, u64* cap, int threads)
{
    if (orc_lde(cols, c, log_n, r, lde, ld, threads)) return -1;
    return orc_merkle(lde, ld, c, log_n + r, h, tree, cap, threads);
}

/* Sec. 2.1 (binning effect): G_B = 2^ceil(log2 G); returns ceil(log2 G). */
uint32_t orc_domain_log2(uint64_t G)
{
    uint32_t k = 0;
    while (((uint64_t)1 << k) < G) k++;
    return k;
}

/* ------------------------------------------------------------------ */
/* FRI commit phase.  The paper's prover uses the default Plonky2 FRI    */
/* setup (Sec. 5, evaluation environment) but prints no FRI formula; the */
/* steps below are the textbook FRI commit phase (Ben-Sasson, Bentov,    */
/* Horesh, Riabzev, ICALP 2018) on the bit-reversed codeword:            */
/*   combine  f_0(x_t) = sum_i alpha^i row_t[i];                         */
/*   fold     f = sum_{i < 2^a} X^i f_i(X^{2^a})  ->  sum_i beta^i f_i;  */
/*   final    coefficients of the last layer's polynomial.               */
/* A layer of size m sits on the coset s * <w_m>; position t holds the   */
/* value at x_t = s * w_m^{bitrev_{log m}(t)}.                           */
/* ------------------------------------------------------------------ */

typedef struct {
    const u64* rows;
    uint32_t ld, c;
    u64 alpha, a0; /* a0 = alpha^e0 */
    int acc;
    u64* out;
} combine_ctx;
static void combine_body(void* vctx, size_t t)
{
    combine_ctx* C = (combine_ctx*)vctx;
    const u64* row = C->rows + t * C->ld;
    u64 s = 0, w = C->a0;
    for (uint32_t i = 0; i < C->c; i++) {
        s = orc_add(s, orc_mul(w, row[i]));
        w = orc_mul(w, C->alpha);
    }
    C->out[t] = C->acc ? orc_add(C->out[t], s) : s;
}

/* out[t] (+)= sum_{i<c} alpha^(e0 + i) * rows[t][i] for t < nrows. */
int orc_fri_combine(const u64* rows, uint32_t ld, uint32_t c, uint64_t nrows, u64 alpha, uint64_t e0,
                    int acc, u64* out, int threads)
{
    combine_ctx C = {rows, ld, c, alpha, orc_pow(alpha, e0), acc, out};
    parallel_for(nrows, threads, combine_body, &C);
    return 0;
}

/* Fold of one coset: output position w of a layer of 2^logm values on
 * shift * <w_m>.  The coset holds positions w*2^a + v (v < 2^a), whose
 * points x_v all square a times to y_w.  With f(x_v) = sum_i x_v^i f_i(y_w),
 * the sum over the coset of f(x_v) x_v^{-i} is 2^a f_i(y_w), so
 *   f_i(y_w) = 2^{-a} sum_v f(x_v) x_v^{-i},  result = sum_i beta^i f_i(y_w).
 * vals[v] = f(x_v). */
u64 orc_fri_fold_coset(const u64* vals, uint32_t logm, u64 shift, uint32_t a, u64 beta, uint64_t w)
{
    uint32_t A = 1u << a;
    u64 w_m = orc_root_of_unity(logm), inv_arity = orc_inv((u64)A);
    u64 xinv[256], xpow[256]; /* x_v^{-1} and x_v^{-i} */
    for (uint32_t v = 0; v < A; v++) {
        xinv[v] = orc_inv(orc_mul(shift, orc_pow(w_m, bitrev((u64)w * A + v, logm))));
        xpow[v] = 1;
    }
    u64 res = 0, bpow = 1;
    for (uint32_t i = 0; i < A; i++) {
        u64 fi = 0;
        for (uint32_t v = 0; v < A; v++) {
            fi = orc_add(fi, orc_mul(vals[v], xpow[v]));
            xpow[v] = orc_mul(xpow[v], xinv[v]);
        }
        fi = orc_mul(fi, inv_arity);
        res = orc_add(res, orc_mul(bpow, fi));
        bpow = orc_mul(bpow, beta);
    }
    return res;
}

typedef struct {
    const u64* f;
    uint32_t logm, a;
    u64 shift, beta;
    u64* out;
} fold_ctx;
static void fold_body(void* vctx, size_t w)
{
    fold_ctx* F = (fold_ctx*)vctx;
    F->out[w] = orc_fri_fold_coset(F->f + (w << F->a), F->logm, F->shift, F->a, F->beta, w);
}

/* One FRI fold of arity 2^a: f has 2^logm values on shift * <w_{2^logm}> in
 * bit-reversed order; out gets 2^(logm - a) values on shift^(2^a) * <...>,
 * also bit-reversed. */
int orc_fri_fold(const u64* f, uint32_t logm, u64 shift, uint32_t a, u64 beta, u64* out, int threads)
{
    if (a == 0 || a > 8 || a > logm) return -1;
    fold_ctx F = {f, logm, a, shift, beta, out};
    parallel_for((size_t)1 << (logm - a), threads, fold_body, &F);
    return 0;
}

/* Coefficients c_i of the polynomial of degree < m whose value at
 * x_t = shift * w_m^{bitrev(t)} is f[t]: by the inverse DFT definition,
 * c_i = m^{-1} shift^{-i} sum_j E_j w_m^{-ij} with E_j = f[bitrev(j)]. */
int orc_fri_interpolate(const u64* f, uint32_t logm, u64 shift, u64* coeffs)
{
    size_t m = (size_t)1 << logm;
    u64 winv = orc_inv(orc_root_of_unity(logm)), minv = orc_inv((u64)m % ORC_P), sinv = orc_inv(shift);
    u64 spow = minv;
    for (size_t i = 0; i < m; i++) {
        u64 s = 0, wi = orc_pow(winv, i), wij = 1;
        for (size_t j = 0; j < m; j++) {
            s = orc_add(s, orc_mul(f[bitrev(j, logm)], wij));
            wij = orc_mul(wij, wi);
        }
        coeffs[i] = orc_mul(s, spow);
        spow = orc_mul(spow, sinv);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Snapshot commitment (Sec. 4.3, "Snapshot Commitments"):             */
/*   hash_{i,j} = Hash(i, j, f_{i,j}, item_{i,j}, v_{i,j}^(0..M-1)),     */
/*   root_i     = MerkleTree(hash_{i,0}, ..., hash_{i,n-1}),            */
/*   hash_i     = Hash(i, mu_i[0..D), root_i),                          */
/*   root_mk    = MerkleTree(hash_0, ..., hash_{nlist-1}),              */
/*   root_cb    = Hash(C_{0,0}, ..., C_{M-1,K-1}) (each C_{m,k} in F^d). */
/* Hash is the Poseidon sponge above; MerkleTree takes the digests as   */
/* its leaves and compresses pairs up to one root.  A slot record is     */
/* stored as [f, item, v^(0), ..., v^(M-1)] (2 + M field elements).      */
/* ------------------------------------------------------------------ */

typedef struct {
    const u64* rec;
    uint32_t n, M;
    u64* out;
} slot_ctx;
static void slot_body(void* vctx, size_t t)
{
    slot_ctx* S = (slot_ctx*)vctx;
    u64 in[2 + 2 + 256];
    in[0] = (u64)(t / S->n); /* i */
    in[1] = (u64)(t % S->n); /* j */
    memcpy(in + 2, S->rec + t * (2 + (size_t)S->M), (2 + (size_t)S->M) * sizeof(u64));
    orc_hash(in, 4 + S->M, S->out + 4 * t);
}

typedef struct {
    const u64* mu;
    const u64* roots;
    uint32_t D;
    u64* out;
    u64* buf;
} cent_ctx;
static void cent_body(void* vctx, size_t i)
{
    cent_ctx* C = (cent_ctx*)vctx;
    size_t L = 1 + (size_t)C->D + 4;
    u64* in = (u64*)malloc(L * sizeof(u64));
    in[0] = (u64)i;
    memcpy(in + 1, C->mu + i * C->D, (size_t)C->D * sizeof(u64));
    memcpy(in + 1 + C->D, C->roots + 4 * i, 4 * sizeof(u64));
    orc_hash(in, (uint32_t)L, C->out + 4 * i);
    free(in);
}

/* Root of the Merkle tree whose 2^log_leaves leaves are the given digests. */
static int digest_tree_root(const u64* leaves, uint32_t log_leaves, u64* root, int threads)
{
    size_t cnt = (size_t)1 << log_leaves;
    u64* level = (u64*)malloc(cnt * 4 * sizeof(u64));
    if (!level) return -1;
    memcpy(level, leaves, cnt * 4 * sizeof(u64));
    while (cnt > 1) {
        u64* next = (u64*)malloc((cnt / 2) * 4 * sizeof(u64));
        if (!next) {
            free(level);
            return -1;
        }
        orc_merkle_level(level, cnt / 2, next, threads);
        free(level);
        level = next;
        cnt /= 2;
    }
    memcpy(root, level, 4 * sizeof(u64));
    free(level);
    return 0;
}

typedef struct {
    const u64* leaves;
    uint32_t log_n;
    u64* roots;
    int failed;
} list_ctx;
/* root_i of one list: its own tree, built serially (lists run in parallel). */
static void list_body(void* vctx, size_t i)
{
    list_ctx* L = (list_ctx*)vctx;
    if (digest_tree_root(L->leaves + (i << L->log_n) * 4, L->log_n, L->roots + 4 * i, 1)) L->failed = 1;
}

/* Slot leaf digests [nlist * n][4] (list-major). */
int orc_snapshot_slot_leaves(const u64* records, uint32_t nlist, uint32_t n, uint32_t M, u64* out, int threads)
{
    if (!params() || M > 256) return -1;
    slot_ctx S = {records, n, M, out};
    parallel_for((size_t)nlist * n, threads, slot_body, &S);
    return 0;
}

/* list_roots [nlist][4], centroid digests [nlist][4], root_mk [4], root_cb [4].
 * nlist and n are powers of two. */
int orc_snapshot_commit(const u64* records, uint32_t log_nlist, uint32_t log_n, uint32_t M, const u64* mu,
                        uint32_t D, const u64* codebooks, uint32_t K, uint32_t d, u64* list_roots,
                        u64* cent_digests, u64* root_mk, u64* root_cb, int threads)
{
    if (!params() || M > 256) return -1;
    size_t nlist = (size_t)1 << log_nlist, n = (size_t)1 << log_n;
    u64* leaves = (u64*)malloc(nlist * n * 4 * sizeof(u64));
    if (!leaves) return -1;
    orc_snapshot_slot_leaves(records, (uint32_t)nlist, (uint32_t)n, M, leaves, threads);
    list_ctx Lc = {leaves, log_n, list_roots, 0};
    parallel_for(nlist, threads, list_body, &Lc);
    free(leaves);
    if (Lc.failed) return -1;
    cent_ctx C = {mu, list_roots, D, cent_digests, NULL};
    parallel_for(nlist, threads, cent_body, &C);
    if (digest_tree_root(cent_digests, log_nlist, root_mk, threads)) return -1;
    orc_hash(codebooks, M * K * d, root_cb);
    return 0;
}

/* root_i of one list from its n = 2^log_n records, for list index i. */
int orc_snapshot_list_root(const u64* list_records, uint64_t i, uint32_t log_n, uint32_t M, u64* root)
{
    if (!params() || M > 256) return -1;
    size_t n = (size_t)1 << log_n;
    u64* leaves = (u64*)malloc(n * 4 * sizeof(u64));
    if (!leaves) return -1;
    u64 in[2 + 2 + 256];
    for (size_t j = 0; j < n; j++) {
        in[0] = i;
        in[1] = (u64)j;
        memcpy(in + 2, list_records + j * (2 + (size_t)M), (2 + (size_t)M) * sizeof(u64));
        orc_hash(in, 4 + M, leaves + 4 * j);
    }
    int rc = digest_tree_root(leaves, log_n, root, 1);
    free(leaves);
    return rc;
}

/* hash_i = Hash(i, mu_i, root_i). */
void orc_snapshot_centroid_digest(uint64_t i, const u64* mu_i, uint32_t D, const u64* root_i, u64* out)
{
    u64* in = (u64*)malloc((1 + (size_t)D + 4) * sizeof(u64));
    in[0] = i;
    memcpy(in + 1, mu_i, (size_t)D * sizeof(u64));
    memcpy(in + 1 + D, root_i, 4 * sizeof(u64));
    orc_hash(in, 1 + D + 4, out);
    free(in);
}

/* ------------------------------------------------------------------ */
/* Multiset equality gadget (Sec. 4.5, set-oriented gadgets).          */
/*   Compress(x; beta) = sum_k x_k beta^k over a tuple of T components; */
/*   SetEq(X, Y): prod_i (alpha - x_i) = prod_i (alpha - y_i).           */
/* The prover's grand-product column (the partial products of a        */
/* PLONK-style permutation argument) is                                 */
/*   Z_0 = 1,  Z_{i+1} = Z_i (alpha - x_i) / (alpha - y_i),             */
/* so Z_L = 1 exactly when the two products agree.  Returns 1 (and      */
/* leaves z undefined) if some alpha - y_i is zero.                      */
/* ------------------------------------------------------------------ */

u64 orc_compress_tuple(const u64* x, uint32_t T, u64 beta)
{
    u64 s = 0, bp = 1;
    for (uint32_t k = 0; k < T; k++) {
        s = orc_add(s, orc_mul(x[k], bp));
        bp = orc_mul(bp, beta);
    }
    return s;
}

int orc_seteq_partial_products(const u64* X, const u64* Y, uint64_t L, uint32_t T, u64 alpha, u64 beta, u64* z)
{
    z[0] = 1;
    for (uint64_t i = 0; i < L; i++) {
        u64 num = orc_sub(alpha, orc_compress_tuple(X + i * T, T, beta));
        u64 den = orc_sub(alpha, orc_compress_tuple(Y + i * T, T, beta));
        if (den == 0) return 1;
        z[i + 1] = orc_mul(z[i], orc_mul(num, orc_inv(den)));
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* FRI over the quadratic extension F_p[u] / (u^2 - 7).  Plonky2's       */
/* default FRI draws its challenges from a degree-2 extension (§5 names  */
/* the default configuration); 7 generates F_p^*, so it is a quadratic   */
/* non-residue and u^2 - 7 is irreducible.  An element is (re, im) =     */
/* re + im u.  The LDE columns stay in F_p; the combination, the layers  */
/* and the final coefficients are extension elements.                    */
/* ------------------------------------------------------------------ */

#define ORC_EXT_W 7ULL

static void ext_mul(const u64* a, const u64* b, u64* out)
{
    u64 re = orc_add(orc_mul(a[0], b[0]), orc_mul(ORC_EXT_W, orc_mul(a[1], b[1])));
    u64 im = orc_add(orc_mul(a[0], b[1]), orc_mul(a[1], b[0]));
    out[0] = re;
    out[1] = im;
}

/* 1 / (re + im u) = (re - im u) / (re^2 - 7 im^2). */
static void ext_inv(const u64* a, u64* out)
{
    u64 n = orc_sub(orc_mul(a[0], a[0]), orc_mul(ORC_EXT_W, orc_mul(a[1], a[1])));
    u64 ni = orc_inv(n);
    out[0] = orc_mul(a[0], ni);
    out[1] = orc_mul(orc_sub(0, a[1]), ni);
}

void orc_ext_mul(const u64* a, const u64* b, u64* out) { ext_mul(a, b, out); }
void orc_ext_inv(const u64* a, u64* out) { ext_inv(a, out); }

typedef struct {
    const u64* rows;
    uint32_t ld, c;
    u64 alpha[2], a0[2];
    int acc;
    u64* out;
} combine_ext_ctx;
static void combine_ext_body(void* vctx, size_t t)
{
    combine_ext_ctx* C = (combine_ext_ctx*)vctx;
    const u64* row = C->rows + t * C->ld;
    u64 s[2] = {0, 0}, w[2] = {C->a0[0], C->a0[1]};
    for (uint32_t i = 0; i < C->c; i++) {
        s[0] = orc_add(s[0], orc_mul(w[0], row[i]));
        s[1] = orc_add(s[1], orc_mul(w[1], row[i]));
        u64 nw[2];
        ext_mul(w, C->alpha, nw);
        w[0] = nw[0];
        w[1] = nw[1];
    }
    if (C->acc) {
        C->out[2 * t] = orc_add(C->out[2 * t], s[0]);
        C->out[2 * t + 1] = orc_add(C->out[2 * t + 1], s[1]);
    } else {
        C->out[2 * t] = s[0];
        C->out[2 * t + 1] = s[1];
    }
}

/* out[t] (+)= sum_{i<c} alpha^(e0+i) rows[t][i], alpha and out in F_p^2. */
int orc_fri_combine_ext(const u64* rows, uint32_t ld, uint32_t c, uint64_t nrows, const u64* alpha, uint64_t e0,
                        int acc, u64* out, int threads)
{
    combine_ext_ctx C;
    C.rows = rows;
    C.ld = ld;
    C.c = c;
    C.alpha[0] = alpha[0];
    C.alpha[1] = alpha[1];
    C.a0[0] = 1;
    C.a0[1] = 0;
    for (uint64_t k = 0; k < e0; k++) {
        u64 nw[2];
        ext_mul(C.a0, alpha, nw);
        C.a0[0] = nw[0];
        C.a0[1] = nw[1];
    }
    C.acc = acc;
    C.out = out;
    parallel_for(nrows, threads, combine_ext_body, &C);
    return 0;
}

/* The coset fold of orc_fri_fold_coset with extension values and challenge:
 * f_i(y_w) = 2^-a sum_v f(x_v) x_v^-i (x_v in F_p), result = sum_i beta^i f_i. */
void orc_fri_fold_coset_ext(const u64* vals /* [2^a][2] */, uint32_t logm, u64 shift, uint32_t a, const u64* beta,
                            uint64_t w, u64* out)
{
    uint32_t A = 1u << a;
    u64 w_m = orc_root_of_unity(logm), inv_arity = orc_inv((u64)A);
    u64 xinv[256], xpow[256];
    for (uint32_t v = 0; v < A; v++) {
        xinv[v] = orc_inv(orc_mul(shift, orc_pow(w_m, bitrev((u64)w * A + v, logm))));
        xpow[v] = 1;
    }
    u64 res[2] = {0, 0}, bpow[2] = {1, 0};
    for (uint32_t i = 0; i < A; i++) {
        u64 fi[2] = {0, 0};
        for (uint32_t v = 0; v < A; v++) {
            fi[0] = orc_add(fi[0], orc_mul(vals[2 * v], xpow[v]));
            fi[1] = orc_add(fi[1], orc_mul(vals[2 * v + 1], xpow[v]));
            xpow[v] = orc_mul(xpow[v], xinv[v]);
        }
        fi[0] = orc_mul(fi[0], inv_arity);
        fi[1] = orc_mul(fi[1], inv_arity);
        u64 t[2];
        ext_mul(bpow, fi, t);
        res[0] = orc_add(res[0], t[0]);
        res[1] = orc_add(res[1], t[1]);
        ext_mul(bpow, beta, t);
        bpow[0] = t[0];
        bpow[1] = t[1];
    }
    out[0] = res[0];
    out[1] = res[1];
}

typedef struct {
    const u64* f;
    uint32_t logm, a;
    u64 shift, beta[2];
    u64* out;
} fold_ext_ctx;
static void fold_ext_body(void* vctx, size_t w)
{
    fold_ext_ctx* F = (fold_ext_ctx*)vctx;
    orc_fri_fold_coset_ext(F->f + 2 * (w << F->a), F->logm, F->shift, F->a, F->beta, w, F->out + 2 * w);
}

int orc_fri_fold_ext(const u64* f, uint32_t logm, u64 shift, uint32_t a, const u64* beta, u64* out, int threads)
{
    if (a == 0 || a > 8 || a > logm) return -1;
    fold_ext_ctx F = {f, logm, a, shift, {beta[0], beta[1]}, out};
    parallel_for((size_t)1 << (logm - a), threads, fold_ext_body, &F);
    return 0;
}
