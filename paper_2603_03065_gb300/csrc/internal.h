// Declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace v3c {

typedef uint64_t u64;
typedef uint32_t u32;

// Twiddle and scale tables of one (log_n, rate_bits) shape, resident in HBM.
// The LDE of n = n1 * n2 rows into N = n * 2^r rows runs in three stages:
//   A  per column and i2 < n2: inverse DFT of size n1 over x[i2 + n2*i1],
//      then twiddle w_n^-(i2*k1)                         -> Y[k1][i2]
//   B  per column and k1 < n1: inverse DFT of size n2 over Y[k1][.] gives the
//      coefficients a_{k1 + n1*k2}.  Scale them by 7^j / n.  The zero-padded
//      forward DFT of size M = n2 * 2^r follows, then the twiddle
//      w_N^(k1*q)                                        -> Z[k1][q]
//   C  per column and q < M: forward DFT of size n1 over Z[.][q] gives
//      E_{q + M*s}, written to committed rows bitrev_M(q)*n1 + bitrev_n1(s).
// With n1 = 1, stages A and C vanish and B writes the rows itself.
struct Plan {
    u32 log_n, r, log_n1, log_n2, log_M, log_N;
    // The coset is g * <w_N> with g = 7 * gshift, and the scale table holds
    // g^j * sfac: gshift = 1, sfac = n^-1 for the LDE of columns.
    u64 gshift, sfac;
    const u64* twa;      // [n1][n2]: w_n^-(k1*i2)                     (n1 > 1)
    const u64* scale;    // [n1][n2]: g^(k1 + n1*bitrev_n2(t)) * sfac, by position t
    const u64* pw_N;     // [3][512]: w_N^(j * 2^(9 level))              (n1 > 1)
    const u64* rinv_n1;  // [n1]:     w_n1^-j
    const u64* rinv_n2;  // [n2/2]:   w_n2^-j
    const u64* rfwd_M;   // [M/2]:    w_M^j
    const u64* rfwd_n1;  // [n1]:     w_n1^j
};

// One LDE job: c columns of one shape.
struct LdeJob {
    Plan plan;
    const u64* x;  // [c][n]
    u64* Y;        // [c][n]   scratch (n1 > 1)
    u64* Z;        // [c][N]   scratch (n1 > 1)
    u64* lde;      // [N][ld]
    u32 c, ld;
    u32 vec_ok;    // lde 16-byte aligned and ld even
    u32 a_cols;    // stage A: i2 columns per CTA (power of two, <= n2)
    u32 c_q;       // Z block: q values per block (power of two, <= M)
    u32 c_qc;      // stage C: q values per CTA (power of two, <= c_q)
    u32 kcap;      // largest radix exponent of the in-register DFT passes (1..4)
    u32 wcols;     // columns writable from lde: ld for a whole matrix, fewer for a column chunk
    u32 mode;      // kLdeFromColumns, kCoeffsOut or kLdeFromCoeffs
    u64 cscale;    // kCoeffsOut: n^-1, applied to the unnormalised inverse DFT
};

// LdeJob.mode.  kLdeFromColumns: the LDE of the input columns x (stages A,
// B, C).  kCoeffsOut: the interpolant's coefficients a = iNTT_n(x), written
// in natural order to `lde` as [c][n] (stage A and the inverse half of
// stage B).  kLdeFromCoeffs: x holds coefficients [c][n] in natural order and
// the LDE is evaluated from them (the forward half of stage B, and stage
// C); the plan's scale table then carries no n^-1.
constexpr u32 kLdeFromColumns = 0;
constexpr u32 kCoeffsOut = 1;
constexpr u32 kLdeFromCoeffs = 2;

// Tile choice of one (log_n, rate_bits) shape, from the autotuner.
struct TuneEntry {
    u32 a_cols, c_q, c_qc, kcap, h_threads;
};

// One Merkle job: leaf hashes then tree levels up to the cap.
struct TreeJob {
    const u64* rows;  // [N][ld]
    u64* tree;        // level-major below the cap (may be null if log_N == h)
    u64* cap;         // [2^h][4]
    u32 ld, width, log_N, h;
    u32 vec_ok;       // rows 16-byte aligned and ld even
    u32 pad;
};

// Work decomposition of one stage over a list of jobs: job j owns items
// [first[j], first[j+1]).  A persistent grid walks the items.
struct StageList {
    const u32* first;  // device [njobs + 1]
    u32 njobs;
    u32 total;
};

// Tile parameters (picked per shape by the autotuner, or defaults).
struct Tiles {
    u32 a_threads, a_cols;   // stage A: threads, i2 columns per CTA
    u32 b_threads;           // stage B
    u32 c_threads, c_q;      // stage C: threads, q values per CTA
    u32 h_threads;           // leaf hash threads per CTA
    u32 m_threads;           // Merkle threads per CTA
};
Tiles default_tiles();
// Per-job tile choice (stage A i2 columns, stage C / Z q-blocking) from the plan.
void lde_job_tiles(LdeJob& j);
// Applies an autotuned choice if it is valid for the job's plan.
bool lde_job_apply_tune(LdeJob& j, const TuneEntry& t);

// Stage launchers (ntt.cu / hash.cu).  Each enqueues one launch on `s`.
cudaError_t build_plan_tables(Plan& p, u64* base, cudaStream_t s);
size_t plan_table_words(u32 log_n, u32 r);
void plan_split(u32 log_n, u32 r, u32& log_n1, u32& log_n2);

u32 stage_a_items(const LdeJob& j, const Tiles& t);
u32 stage_b_items(const LdeJob& j);
u32 stage_c_items(const LdeJob& j, const Tiles& t);
size_t stage_a_smem(const LdeJob& j, const Tiles& t);
size_t stage_b_smem(const LdeJob& j);
size_t stage_c_smem(const LdeJob& j, const Tiles& t);

cudaError_t launch_stage_a(const LdeJob* d_jobs, StageList l, size_t smem, const Tiles& t, int grid,
                           cudaStream_t s);
// spec: every job of the launch satisfies lde_job_spec (stage B's specialised kernel).
cudaError_t launch_stage_b(const LdeJob* d_jobs, StageList l, size_t smem, const Tiles& t, int grid,
                           cudaStream_t s, bool spec = false);
cudaError_t launch_stage_c(const LdeJob* d_jobs, StageList l, size_t smem, const Tiles& t, int grid,
                           cudaStream_t s);
// An LDE of columns with the 2^10 x 2^3 plan and the default tiles.
bool lde_job_spec(const LdeJob& j);

u32 leaf_items(const TreeJob& j, const Tiles& t);
cudaError_t launch_leaf_hash(const TreeJob* d_jobs, StageList l, const Tiles& t, int grid, cudaStream_t s);
// Merkle levels [lev0+1, lev0+nlev] of each job (only jobs with top > lev0).
u32 merkle_items(const TreeJob& j, u32 lev0, const Tiles& t);
cudaError_t launch_merkle(const TreeJob* d_jobs, StageList l, u32 lev0, u32 nlev, const Tiles& t, int grid,
                          cudaStream_t s);
// Warp-per-node form for small levels, where one compression's latency sets
// the time of a level: one warp per compression, kMerkleWarps nodes of
// level lev0+1 per CTA, up to kMerkleWarpLevels levels folded in shared
// memory.  Used once a level has at most kMerkleWarpMaxNodes nodes (one CTA
// of 1024 threads per SM, one wave).
constexpr u32 kMerkleWarps = 32;
constexpr u32 kMerkleWarpLevels = 6;
constexpr u64 kMerkleWarpMaxNodes = 4096;
u32 merkle_warp_items(const TreeJob& j, u32 lev0);
cudaError_t launch_merkle_warp(const TreeJob* d_jobs, StageList l, u32 lev0, u32 nlev, int grid, cudaStream_t s);

cudaError_t launch_validate(const u64* x, u64 count, u32* d_flag, cudaStream_t s);
cudaError_t launch_int_peak(u64* out, int grid, int threads, u32 iters, int wide, cudaStream_t s);

int max_smem_optin();
int num_sms();

}  // namespace v3c
