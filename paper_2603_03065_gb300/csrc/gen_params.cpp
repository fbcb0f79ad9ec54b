// Build-time generator of the Poseidon-w12 parameters compiled into the
// kernels.  It writes a header with the round constants and the first row of
// the circulant MDS matrix.
//
// Derivation (the paper names Poseidon as its hash, Sec. 4.3, but fixes no
// parameters; this is the library's own definition):
//   * Stream: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).  Each step adds
//     0x9E3779B97F4A7C15 to the state.  The output is the new state mixed by
//     the two multiply/xor-shift rounds of the published finaliser.  The seed
//     is the ASCII bytes "V3DBPOS1" read big-endian.
//   * Round constants RC[round][lane], round-major: consecutive draws, each
//     kept only if it is below p.
//   * MDS: the following draws fill candidate rows m[0..11] with (draw & 63),
//     skipping zeros.  The matrix is M[i][j] = m[(j - i) mod 12].  The first
//     candidate with every square minor nonzero mod p is used.
//
// The minors are checked by expansion along the lowest-numbered column of
// each column subset.  The minors of each size are memoised and indexed by
// combinatorial rank.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace {

typedef unsigned __int128 u128;
constexpr uint64_t kP = 0xFFFFFFFF00000001ULL;
constexpr int kW = 12;
constexpr int kRounds = 30;

struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        s += 0x9E3779B97F4A7C15ULL;
        uint64_t z = s;
        z ^= z >> 30;
        z *= 0xBF58476D1CE4E5B9ULL;
        z ^= z >> 27;
        z *= 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
};

uint64_t fmul(uint64_t a, uint64_t b) { return (uint64_t)((u128)a * b % kP); }
uint64_t fadd(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a + b) % kP); }
uint64_t fneg(uint64_t a) { return a ? kP - a : 0; }

// Combinatorial rank of a subset (bitmask over 12 items) among subsets of
// the same size, by the combinatorial number system.
struct Ranker {
    uint32_t binom[kW + 1][kW + 1];
    Ranker()
    {
        memset(binom, 0, sizeof binom);
        for (int n = 0; n <= kW; n++) {
            binom[n][0] = 1;
            for (int k = 1; k <= n; k++) binom[n][k] = binom[n - 1][k - 1] + (k <= n - 1 ? binom[n - 1][k] : 0);
        }
    }
    uint32_t rank(uint32_t mask) const
    {
        uint32_t r = 0;
        int k = 0;
        for (int i = 0; i < kW; i++)
            if (mask >> i & 1) {
                k++;
                r += binom[i][k];
            }
        return r;
    }
};

// True iff every square minor of A (12x12, entries < p) is nonzero mod p.
bool all_minors_nonzero(const uint64_t A[kW][kW])
{
    Ranker rk;
    std::vector<uint32_t> by_size[kW + 1];
    for (uint32_t m = 1; m < (1u << kW); m++) by_size[__builtin_popcount(m)].push_back(m);
    std::vector<uint64_t> prev, cur;
    // size 1
    size_t n1 = by_size[1].size();
    prev.assign(n1 * n1, 0);
    for (uint32_t rm : by_size[1])
        for (uint32_t cm : by_size[1]) {
            uint64_t v = A[__builtin_ctz(rm)][__builtin_ctz(cm)];
            if (v == 0) return false;
            prev[rk.rank(rm) * n1 + rk.rank(cm)] = v;
        }
    size_t nprev = n1;
    for (int k = 2; k <= kW; k++) {
        size_t nk = by_size[k].size();
        cur.assign(nk * nk, 0);
        for (uint32_t cm : by_size[k]) {
            int c0 = __builtin_ctz(cm);           // expand along this column
            uint32_t crest = rk.rank(cm & ~(1u << c0));
            uint32_t cr = rk.rank(cm);
            for (uint32_t rm : by_size[k]) {
                uint64_t acc = 0;
                int pos = 0;
                for (int r = 0; r < kW; r++) {
                    if (!(rm >> r & 1)) continue;
                    uint64_t sub = prev[rk.rank(rm & ~(1u << r)) * nprev + crest];
                    uint64_t term = fmul(A[r][c0], sub);
                    acc = fadd(acc, (pos & 1) ? fneg(term) : term);
                    pos++;
                }
                if (acc == 0) return false;
                cur[rk.rank(rm) * nk + cr] = acc;
            }
        }
        prev.swap(cur);
        nprev = nk;
    }
    return true;
}

uint64_t fsub(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a + kP - b) % kP); }
uint64_t fpow(uint64_t a, uint64_t e)
{
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = fmul(r, a);
        a = fmul(a, a);
        e >>= 1;
    }
    return r;
}
uint64_t finv(uint64_t a) { return fpow(a, kP - 2); }

constexpr int kN = kW - 1;  // the 11x11 lower-right block
constexpr int kRF = 4;      // full rounds before and after the partial rounds
constexpr int kRP = 22;     // partial rounds

// Gauss-Jordan inverse of an 11x11 matrix mod p; false if singular.
bool inverse11(const uint64_t A[kN][kN], uint64_t out[kN][kN])
{
    uint64_t m[kN][2 * kN];
    for (int i = 0; i < kN; i++)
        for (int j = 0; j < 2 * kN; j++) m[i][j] = j < kN ? A[i][j] : (j - kN == i ? 1 : 0);
    for (int c = 0; c < kN; c++) {
        int piv = -1;
        for (int r = c; r < kN; r++)
            if (m[r][c]) {
                piv = r;
                break;
            }
        if (piv < 0) return false;
        for (int j = 0; j < 2 * kN; j++) std::swap(m[c][j], m[piv][j]);
        uint64_t iv = finv(m[c][c]);
        for (int j = 0; j < 2 * kN; j++) m[c][j] = fmul(m[c][j], iv);
        for (int r = 0; r < kN; r++) {
            if (r == c || !m[r][c]) continue;
            uint64_t f = m[r][c];
            for (int j = 0; j < 2 * kN; j++) m[r][j] = fsub(m[r][j], fmul(f, m[c][j]));
        }
    }
    for (int i = 0; i < kN; i++)
        for (int j = 0; j < kN; j++) out[i][j] = m[i][kN + j];
    return true;
}

// Constants of the equivalent fast form of the 22 partial rounds.
//
// A partial round is x <- M S(x + c) with the S-box on lane 0 only.
//  * Constants: the lanes 1..11 of c pass the S-box unchanged, so
//    M S(x + c) = M S(x + c_0 e_0) + M (0, c_1..11).  The second term is
//    carried forward into the next round's constant.  Each partial round
//    then adds one scalar a_k to lane 0, and the leftover vector joins the
//    constants of the first full round after the partial rounds.
//  * Matrices: the map F_k(x) = ((x_0 + a_k)^7, x_1..11) commutes with any
//    D = diag(1, A).  Going backwards from the last partial round,
//    N = Ms_k D_k with D_k = diag(1, N_11) and
//    Ms_k = [[N_00, N_01 N_11^-1], [N_10, I]], and the next N is D_k M.
//    The last D_0 is applied once, right after the MDS of the last full
//    round before the partial rounds.
// Row 0 of every N equals row 0 of M, so Ms_k[0][0] = m_0 for every k.
struct FastParams {
    uint64_t a[kRP];
    uint64_t v[kRP][kN];  // Ms_k row 0, columns 1..11
    uint64_t w[kRP][kN];  // Ms_k column 0, rows 1..11
    uint64_t a0[kN][kN];  // D_0's 11x11 block
    uint64_t rc_after[kW];  // constants of the first full round after the partial rounds
};

bool derive_fast(const uint64_t M[kW][kW], const uint64_t rc[kRounds][kW], FastParams& fp)
{
    uint64_t chat[kW];
    for (int i = 0; i < kW; i++) chat[i] = rc[kRF][i];
    for (int k = 0; k < kRP; k++) {
        fp.a[k] = chat[0];
        uint64_t d[kW];
        for (int i = 0; i < kW; i++) {
            uint64_t acc = 0;
            for (int j = 1; j < kW; j++) acc = fadd(acc, fmul(M[i][j], chat[j]));
            d[i] = acc;
        }
        const uint64_t* next = k + 1 < kRP ? rc[kRF + k + 1] : rc[kRF + kRP];
        for (int i = 0; i < kW; i++) chat[i] = fadd(next[i], d[i]);
    }
    for (int i = 0; i < kW; i++) fp.rc_after[i] = chat[i];
    uint64_t N[kW][kW];
    memcpy(N, M, sizeof N);
    for (int k = kRP - 1; k >= 0; k--) {
        uint64_t A[kN][kN], Ai[kN][kN];
        for (int i = 0; i < kN; i++)
            for (int j = 0; j < kN; j++) A[i][j] = N[1 + i][1 + j];
        if (!inverse11(A, Ai)) return false;
        for (int j = 0; j < kN; j++) {
            uint64_t acc = 0;
            for (int i = 0; i < kN; i++) acc = fadd(acc, fmul(N[0][1 + i], Ai[i][j]));
            fp.v[k][j] = acc;
            fp.w[k][j] = N[1 + j][0];
        }
        if (N[0][0] != M[0][0]) return false;
        if (k == 0) {
            memcpy(fp.a0, A, sizeof A);
            break;
        }
        uint64_t Nn[kW][kW];
        for (int c = 0; c < kW; c++) Nn[0][c] = M[0][c];
        for (int i = 0; i < kN; i++)
            for (int c = 0; c < kW; c++) {
                uint64_t acc = 0;
                for (int j = 0; j < kN; j++) acc = fadd(acc, fmul(A[i][j], M[1 + j][c]));
                Nn[1 + i][c] = acc;
            }
        memcpy(N, Nn, sizeof N);
    }
    return true;
}

uint64_t sbox(uint64_t x)
{
    uint64_t x2 = fmul(x, x), x3 = fmul(x2, x), x4 = fmul(x2, x2);
    return fmul(x3, x4);
}

void mds_mul(const uint64_t M[kW][kW], uint64_t s[kW])
{
    uint64_t t[kW];
    for (int i = 0; i < kW; i++) {
        uint64_t acc = 0;
        for (int j = 0; j < kW; j++) acc = fadd(acc, fmul(M[i][j], s[j]));
        t[i] = acc;
    }
    memcpy(s, t, sizeof t);
}

void permute_plain(const uint64_t M[kW][kW], const uint64_t rc[kRounds][kW], uint64_t s[kW])
{
    for (int r = 0; r < kRounds; r++) {
        for (int i = 0; i < kW; i++) s[i] = fadd(s[i], rc[r][i]);
        bool full = r < kRF || r >= kRF + kRP;
        for (int i = 0; i < (full ? kW : 1); i++) s[i] = sbox(s[i]);
        mds_mul(M, s);
    }
}

void permute_fast(const uint64_t M[kW][kW], const uint64_t rc[kRounds][kW], const FastParams& fp, uint64_t s[kW])
{
    for (int r = 0; r < kRF; r++) {
        for (int i = 0; i < kW; i++) s[i] = sbox(fadd(s[i], rc[r][i]));
        mds_mul(M, s);
    }
    uint64_t t[kN];
    for (int i = 0; i < kN; i++) {
        uint64_t acc = 0;
        for (int j = 0; j < kN; j++) acc = fadd(acc, fmul(fp.a0[i][j], s[1 + j]));
        t[i] = acc;
    }
    for (int i = 0; i < kN; i++) s[1 + i] = t[i];
    for (int k = 0; k < kRP; k++) {
        uint64_t x0 = sbox(fadd(s[0], fp.a[k]));
        uint64_t n0 = fmul(M[0][0], x0);
        for (int j = 0; j < kN; j++) n0 = fadd(n0, fmul(fp.v[k][j], s[1 + j]));
        for (int j = 0; j < kN; j++) s[1 + j] = fadd(s[1 + j], fmul(fp.w[k][j], x0));
        s[0] = n0;
    }
    for (int r = kRF + kRP; r < kRounds; r++) {
        const uint64_t* c = r == kRF + kRP ? fp.rc_after : rc[r];
        for (int i = 0; i < kW; i++) s[i] = sbox(fadd(s[i], c[i]));
        mds_mul(M, s);
    }
}

void emit_array(FILE* f, const char* name, const uint64_t* v, int n)
{
    fprintf(f, "#define %s {", name);
    for (int i = 0; i < n; i++) fprintf(f, "%s%s0x%016llxull", i ? ", " : "", i % 4 == 0 ? "\\\n  " : "", (unsigned long long)v[i]);
    fprintf(f, "}\n");
}

}  // namespace

int main(int argc, char** argv)
{
    if (argc != 2) {
        fprintf(stderr, "usage: %s out_header\n", argv[0]);
        return 2;
    }
    uint64_t seed = 0;
    for (char ch : std::string("V3DBPOS1")) seed = (seed << 8) | (uint8_t)ch;
    SplitMix sm{seed};
    static uint64_t rc[kRounds][kW];
    for (int r = 0; r < kRounds; r++)
        for (int i = 0; i < kW; i++) {
            uint64_t d;
            do d = sm.next();
            while (d >= kP);
            rc[r][i] = d;
        }
    uint64_t row[kW];
    int tries = 0;
    for (;;) {
        tries++;
        if (tries > 100000) {
            fprintf(stderr, "gen_params: no MDS candidate found\n");
            return 1;
        }
        for (int i = 0; i < kW; i++) {
            uint64_t e;
            do e = sm.next() & 63;
            while (e == 0);
            row[i] = e;
        }
        uint64_t A[kW][kW];
        for (int i = 0; i < kW; i++)
            for (int j = 0; j < kW; j++) A[i][j] = row[(j - i + kW) % kW];
        if (all_minors_nonzero(A)) break;
    }
    uint64_t M[kW][kW];
    for (int i = 0; i < kW; i++)
        for (int j = 0; j < kW; j++) M[i][j] = row[(j - i + kW) % kW];
    static FastParams fp;
    if (!derive_fast(M, rc, fp)) {
        fprintf(stderr, "gen_params: fast partial-round factorisation failed\n");
        return 1;
    }
    // Self-check: the fast form equals the plain round loop on seeded states.
    SplitMix chk{0x5EED5EED5EED5EEDULL};
    for (int t = 0; t < 64; t++) {
        uint64_t a[kW], b[kW];
        for (int i = 0; i < kW; i++) {
            uint64_t d;
            do d = chk.next();
            while (d >= kP);
            a[i] = b[i] = t < 2 ? (t ? kP - 1 : 0) : d;
        }
        permute_plain(M, rc, a);
        permute_fast(M, rc, fp, b);
        if (memcmp(a, b, sizeof a)) {
            fprintf(stderr, "gen_params: fast permutation differs from the plain one\n");
            return 1;
        }
    }
    FILE* f = fopen(argv[1], "w");
    if (!f) {
        perror("gen_params");
        return 1;
    }
    fprintf(f, "// Generated at build time by gen_params.cpp; do not edit.\n");
    fprintf(f, "#pragma once\n#include <stdint.h>\n");
    fprintf(f, "#define V3C_MDS_CANDIDATES %d\n", tries);
    fprintf(f, "#define V3C_MDS_ROW_INIT {");
    for (int i = 0; i < kW; i++) fprintf(f, "%s%lluu", i ? ", " : "", (unsigned long long)row[i]);
    fprintf(f, "}\n#define V3C_RC_INIT {");
    for (int r = 0; r < kRounds; r++) {
        fprintf(f, "%s\\\n  {", r ? "," : "");
        for (int i = 0; i < kW; i++) fprintf(f, "%s0x%016llxull", i ? ", " : "", (unsigned long long)rc[r][i]);
        fprintf(f, "}");
    }
    fprintf(f, "}\n");
    // Fast form of the partial rounds (see derive_fast).
    emit_array(f, "V3C_FAST_A_INIT", fp.a, kRP);
    emit_array(f, "V3C_FAST_V_INIT", &fp.v[0][0], kRP * kN);
    emit_array(f, "V3C_FAST_W_INIT", &fp.w[0][0], kRP * kN);
    emit_array(f, "V3C_FAST_D0_INIT", &fp.a0[0][0], kN * kN);
    emit_array(f, "V3C_FAST_RC_AFTER_INIT", fp.rc_after, kW);
    uint64_t rc_full[2 * kRF][kW];
    for (int r = 0; r < kRF; r++)
        for (int i = 0; i < kW; i++) {
            rc_full[r][i] = rc[r][i];
            rc_full[kRF + r][i] = r == 0 ? fp.rc_after[i] : rc[kRF + kRP + r][i];
        }
    emit_array(f, "V3C_FAST_RC_FULL_INIT", &rc_full[0][0], 2 * kRF * kW);
    // Round constants split into 22-bit limbs (bits 0-21, 22-43, 44-63) for
    // rounds 0..29, plus a zero row 30: the MDS of round r starts its limb
    // accumulators from the constants of round r + 1.
    fprintf(f, "#define V3C_RC_LIMBS_INIT {");
    for (int r = 0; r <= kRounds; r++)
        for (int i = 0; i < kW; i++) {
            uint64_t v = r < kRounds ? rc[r][i] : 0;
            fprintf(f, "%s%s%uu, %uu, %uu", (r || i) ? ", " : "", i == 0 ? "\\\n  " : "",
                    (unsigned)(v & 0x3FFFFF), (unsigned)((v >> 22) & 0x3FFFFF), (unsigned)(v >> 44));
        }
    fprintf(f, "}\n");
    // Round constants for the split MDS (21-bit limbs a = bits 0-20,
    // b = 21-41, c = 42-63), rounds 0..29 plus a zero row 30, all mod 2^32.
    // Limbs a and b (second split): with P_i = a_i + a_(i+6),
    // [P_i + P_(i+3)] (3), [P_i - P_(i+3)] (3), [2 (a_i - a_(i+6))] (6);
    // limb c: [c_i + c_(i+6)] (6), [c_i - c_(i+6)] (6).
    fprintf(f, "#define V3C_RC_SPLIT_INIT {");
    for (int r = 0; r <= kRounds; r++) {
        uint32_t la[kW], lb[kW], lc[kW];
        for (int i = 0; i < kW; i++) {
            uint64_t v = r < kRounds ? rc[r][i] : 0;
            la[i] = (uint32_t)(v & 0x1FFFFF);
            lb[i] = (uint32_t)((v >> 21) & 0x1FFFFF);
            lc[i] = (uint32_t)(v >> 42);
        }
        uint32_t row[36];
        const uint32_t* lab[2] = {la, lb};
        for (int h = 0; h < 2; h++) {
            const uint32_t* l = lab[h];
            uint32_t Pi[6];
            for (int i = 0; i < 6; i++) Pi[i] = l[i] + l[i + 6];
            for (int i = 0; i < 3; i++) {
                row[12 * h + i] = Pi[i] + Pi[i + 3];
                row[12 * h + 3 + i] = Pi[i] - Pi[i + 3];
            }
            for (int i = 0; i < 6; i++) row[12 * h + 6 + i] = 2u * (l[i] - l[i + 6]);
        }
        for (int i = 0; i < 6; i++) {
            row[24 + i] = lc[i] + lc[i + 6];
            row[30 + i] = lc[i] - lc[i + 6];
        }
        for (int k = 0; k < 36; k++)
            fprintf(f, "%s%s%uu", (r || k) ? ", " : "", k % 12 == 0 ? "\\\n  " : "", (unsigned)row[k]);
    }
    fprintf(f, "}\n");
    fclose(f);
    return 0;
}
