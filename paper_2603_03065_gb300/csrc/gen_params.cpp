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
    fclose(f);
    return 0;
}
