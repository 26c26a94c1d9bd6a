// Device side of the B300 BMND denoiser (sm_103a).
//
// Work decomposition.  The reference origins of one array are partitioned into
// tiles: a tile owns the origins r with r_d in [t_d C_d, t_d C_d + C_d).  All
// candidate patches of those references lie in the tile's *region*
// [t_d C_d - rad_d, t_d C_d + C_d - 1 + rad_d + j_d - 1], so one CTA stages the
// region of the guide (and of the observation) in shared memory once and runs
// matching, the group transform, shrinkage, the inverse transform and the
// Kaiser-weighted overlap-add for every reference of the tile out of it.
//
// Aggregation is atomic-free and deterministic: warps accumulate their groups
// into the tile's shared (numerator, weight) region one after another, in
// reference order, handing the turn on with named barriers; each tile then
// writes its region as a partial, and a reduce kernel sums the partials of the
// tiles covering every location in tile order before normalizing
// (Def. "Weighted overlap-add estimate").  The result therefore does not depend
// on scheduling, on the number of jobs in a batched launch, or on timing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace bmnd {

constexpr int KMAXD = 6;     // non-singleton axes handled by the kernels
constexpr int MMAX = 32;     // maximum group size
constexpr int JMAX = 32;     // maximum patch length per axis
constexpr int NW = 8;        // warps per CTA of the stage kernel
constexpr int RPAD = 40;     // floats of padding after every shared region

// DCT table in global memory: orthonormal DCT-II matrices of sizes 1..32 at
// offset (J-1)J(2J-1)/6, then their entrywise squares at +GEN_TOTAL.  Each CTA
// copies the matrices of its patch axes (forward, transposed, squared) into
// shared memory.
constexpr int GEN_TOTAL = 11440;

// Uploads the fast-DCT constants to the constant bank of the current device:
// sec31[N/2 - 1 + n] = 1 / (2 cos(pi (2n+1) / (2N))) for N = 2, 4, ..., 32 and
// scale12[2 log2 N] = sqrt(1/N), scale12[2 log2 N + 1] = sqrt(2/N), N = 1..32.
cudaError_t upload_fast_dct_constants(const float *sec31, const float *scale12);

// Bytes of one warp's shared block: member list, weights, plane sums and the
// members' footprint offsets (4 x MMAX words), nbuf group buffers of M x MS floats (two for
// filtering, one for a second mass-conservation sweep from the synthesis
// cache; their float count rounded up to even), the private footprint (fp
// float2, 8-byte aligned) and, when y and eta are read from global memory
// (lean), the members' global origins (MMAX int64), rounded up to 16.
__host__ __device__ constexpr int warp_bytes(int M, int MS, int fp, int lean, int nbuf = 2) {
  return (4 * MMAX * 4 + ((nbuf * M * MS + 1) & ~1) * 4 + fp * 8 + (lean ? MMAX * 8 : 0) + 15) & ~15;
}

// Floats reserved in shared memory for the four J x J matrices of one patch
// axis -- forward F, synthesis S (F^T for the orthonormal DCT), the entrywise
// square of F and F^T -- rounded up to 4 so that every block starts on a
// 16-byte boundary (the line transforms read rows of sizes divisible by 4 as
// float4).
__host__ __device__ constexpr int mat_block(int J) { return (4 * J * J + 3) & ~3; }

// Per-array geometry of one stage, with singleton axes removed.
struct DGeom {
  int D;
  int P;        // patch entries
  int rows;     // P / jL
  int jL;       // patch length on the last axis
  int LS;       // shared-buffer line stride (jL, padded to odd)
  int MS;       // shared-buffer member stride (rows * LS)
  int region;   // prod RG
  int ntiles;
  int cap;      // prod C: capacity of the per-tile reference list
  int stage;    // 1 hard threshold, 2 Wiener
  int M;        // maximum group size
  int min_group;
  int gtrans;   // 0 Haar, 1 DCT along the group axis
  int wmodel;   // 0 classic, 1 variance, 2 risk
  int wscope;   // 0 patch, 1 group
  int poisson;
  int bias_on;  // stage-1 SSD noise-bias correction active
  float gamma, tau, lambda, s_v, a_power, s_p, var_g;
  int64_t N;
  int64_t L[KMAXD], st[KMAXD], ell[KMAXD];
  int j[KMAXD], rad[KMAXD];
  int C[KMAXD], NT[KMAXD], RG[KMAXD], rst[KMAXD];
  // extents of the staged region's layout: RG, with the last axis padded to
  // an odd length when there are two or more axes (window rows a row stride
  // apart then fall into distinct banks); region and rst follow the layout
  int RGP[KMAXD];
  float kaiser[KMAXD][JMAX];
  // private group footprint (2 rad_d + j_d per axis) used to accumulate a
  // group before merging it into the tile region; fp = 0 disables it
  int fp;
  int FW[KMAXD];
  // lean: only the matching guide is staged in shared memory; the filter
  // reads y (stage 2) and eta (second mass-conservation sweep) from global
  // memory, which leaves room for larger tiles when D >= 3
  int lean;
  // Poisson matching distance of this stage (0 SSD, 1 deviance, 2 Pearson,
  // 3 Anscombe-SSD) and acceptance policy (0 fixed, 1 reference finite-count,
  // 2 candidate-standardized); tau is then in sum units (P d_m) for the fixed
  // policy and t for the standardized one.  mt = t, beta_p = beta_s P,
  // kappa = kappa_s, inv_sp = float(1 / s_P); mom[n] = (mu_m(n), v_m(n)),
  // n = 0..MOMENT_NMAX.  Only the generic (JL = 0) kernels read these.
  int metric, policy;
  int soft;     // stage-1 soft thresholding (Eq. soft-threshold) instead of hard
  // windowed synthesized-domain weights (Sec. 7.3): every coefficient's
  // weight term takes prod_d wsyn[d][q_d], wsyn[d][q] = sum_p DCT_d(q, p)^2
  // kaiser_d(p)^2 (the diagonal of the windowed synthesis metric)
  int wdomain;
  float wsyn[KMAXD][JMAX];
  // leading group-axis planes with the partial shared-source Poisson
  // variance (Sec. 5); 0 = the diagonal model.  Generic kernels only.
  int kex;
  float mt, beta_p, kappa, inv_sp;
  const float2 *mom;
  // Decisions in double precision.  Matching ranks and accepts candidates,
  // and the hard threshold keeps coefficients, by comparisons that the FP32
  // fast path can only take where its error bound separates the two sides;
  // the rest are re-evaluated in double precision with these scalars as
  // the definitions have them: s_P, gamma, the Gaussian bias 2 P sigma^2
  // (0 for Poisson noise), tau, lambda and sigma^2; dct64 holds the
  // orthonormal DCT-II matrices of sizes 1..32 at gen_off(J).  ku bounds the
  // error of an FP32 SSD score per unit of its magnitude (ssd + gamma B);
  // ht_t2 is the largest squared entry of the spatial transform.  exact_ok:
  // stage-1 SSD with s_P a power of two and an integral gamma, where tiles
  // of dyadic data score exactly in FP32.
  double s_p64, gamma64, gbias64, tau64, lambda64, var64;
  const double *dct64;
  float ku, ht_t2;
  int exact_ok;
  // spatial transform of this stage: 0 the orthonormal DCT-II, 1 bior1.5
  // (stage 1 only, App. A) from dense shared-memory matrices; sp64: its
  // double forward matrices (gen_off layout); ht_band: widening of the FP32
  // hard-threshold error band for the dense non-orthonormal transform
  int spatial;
  const double *sp64;
  float ht_band;
  // bsm: the stage kernels keep a patch-sum map of the guide (one float per
  // region position) for the stage-1 noise bias of non-negative tiles
  int bsm;
  // Poisson distances on count data in exact integer arithmetic: pfix
  // holds fixed-point tables (units 2^-32) of the per-entry contributions
  // and the finite-count moments (layout at PFIX_*), and count_tol the
  // relative distance from an integer within which y / s_P is a count.
  const long long *pfix;
  double mt64, beta_p64, kappa64;  // t, beta_s P, kappa_s in double
  // counters of the double-precision decisions (or null): [0] candidates
  // rescored, [1] full double-precision searches, [2] coefficients decided
  // in double precision at the hard threshold
  unsigned long long *diag;
};

// Layout of the transform tables in device memory: the float DCT table
// (2 GEN_TOTAL floats, see above), at float TAB_BIOR the bior1.5 analysis
// matrices and at TAB_BIOR + GEN_TOTAL their synthesis matrices (power-of-two
// sizes, same offsets), and at TAB64_OFFSET bytes the double DCT matrices
// followed by the double bior1.5 analysis matrices (GEN_TOTAL doubles each).
constexpr int TAB_BIOR = 2 * GEN_TOTAL;
constexpr int TAB64_OFFSET = ((4 * GEN_TOTAL * 4) + 255) & ~255;
constexpr int TAB_BYTES = TAB64_OFFSET + 2 * GEN_TOTAL * 8;

constexpr int MOMENT_NMAX = 4096;

// FP32 throughput probe: independent FMA chains per thread
constexpr int FMA_PEAK_CHAINS = 8 * 16;

// Fixed-point tables of a Poisson distance for count data (int64, units
// 2^-32 unless stated): at PFIX_A, indexed by a count K <= PFIX_K:
// deviance K ln(2K), Pearson floor(2^64 / K) (K >= 1), Anscombe
// 2 sqrt(K + 3/8) in units 2^-44; at PFIX_B the deviance's K ln K; at PFIX_MU
// and PFIX_V the moments mu(n), v(n), n <= MOMENT_NMAX.  Counts up to
// PFIX_K / 2 per entry, so pooled counts stay within the tables.
constexpr int PFIX_K = 16384;
constexpr int PFIX_A = 0;
constexpr int PFIX_B = PFIX_K + 1;
constexpr int PFIX_MU = 2 * (PFIX_K + 1);
constexpr int PFIX_V = PFIX_MU + MOMENT_NMAX + 1;
constexpr int PFIX_TOTAL = PFIX_V + MOMENT_NMAX + 1;

struct DJob {
  DGeom g;
  const float *y;      // observation
  const float *guide;  // matching guide and variance-map source (y or pilot)
  float *out;          // stage estimate
  float *eta;          // overlap-add denominator (mass conservation)
  float2 *partial;     // ntiles * region (numerator, weight)
  const int *ref_local;  // ntiles * cap core-local reference indices
  const int *ref_count;  // ntiles
  int *groups;         // ntiles * cap * M region offsets of members (or null)
  int *gcount;         // ntiles * cap group sizes
  int tile_base;       // first tile of this job in a batched grid
  int pad0;
  int64_t vox_base;    // first location of this job in a batched reduce
  // synthesis cache of the first mass-conservation sweep (or null): for the
  // reference r = ref_base[tile] + slot, pcache[(r M + m) P + v] holds entry
  // v of synthesized member m and wcache[r M + m] its weight; r < pcache_refs
  float *pcache;
  float *wcache;
  const int *ref_base;
  int64_t pcache_refs;
};

// Geometry of a reference-coverage map (Sec. 9.3) over the kernel axes:
// array extents L, patch sides j, last valid origins ell and the strides fst
// of the schedule's byte grid of origins (nflags bytes).
struct CovGeom {
  int D, P;
  int64_t N, nflags;
  int64_t L[KMAXD], ell[KMAXD], fst[KMAXD];
  int j[KMAXD];
};

// Schedule geometry on the full (unsqueezed) shape.
struct SGeom {
  int ndim;
  int schedule;   // 0 generated, 1 off, 2 sparse, 3 balanced
  int passes;
  int D;          // kernel axes
  double rho;
  int64_t Z[8], ell[8];
  int j[8], h[8];
  int kax[8];     // kernel axis of each full axis (-1 if singleton)
  int64_t fst[KMAXD];  // strides of the origin grid over kernel axes
  int64_t nslots;
};

}  // namespace bmnd
