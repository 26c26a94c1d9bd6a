// Host side of the B300 BMND denoiser: argument checks, per-array planning
// (tile geometry, scratch layout, shared-memory budget), launches, and the C
// ABI declared in include/bmnd.h.
#include "../../include/bmnd.h"
#include "bmnd_kernels.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace bmnd {
typedef void (*stage_fn)(const DJob *, int, int, int, const float *, int *);
stage_fn select_stage_kernel(int D, int jL, int kb, int minb, int stage);
void launch_reduce(int D, const DJob *jobs, int njobs, int64_t total, int write_eta, int grid,
                   cudaStream_t st);
void launch_export(int D, const DJob *jobs, int ntiles, const int64_t *tile_off, int64_t *origins,
                   int64_t *groups, int32_t *counts, int64_t cap, cudaStream_t st);
void launch_sched(const SGeom &s, unsigned char *flags, const DJob *jobs, int ntiles, int *ref_local,
                  int *ref_count, cudaStream_t st);
void launch_ref_base(const int *count, int ntiles, int *ref_base, cudaStream_t st);
void launch_fma_peak(float *out, int blocks, int threads, int iters);
void launch_sched_mark(const SGeom &s, unsigned char *flags, cudaStream_t st);
void launch_coverage(const CovGeom &c, const unsigned char *flags, int32_t *cov, unsigned long long *sums,
                     cudaStream_t st);
cudaError_t set_stage_smem(stage_fn f, int bytes);
}  // namespace bmnd

using namespace bmnd;

struct bmnd_ctx {
  int device = 0;
  size_t budget = 0;
  char err[512] = {0};
  void *arena = nullptr;
  size_t arena_size = 0;
  float *tab = nullptr;        // generic DCT matrices, sizes 1..32 (+ squares), then the double matrices
  const double *tab64 = nullptr;  // double matrices inside the tab allocation (TAB64_OFFSET)
  unsigned long long *diag = nullptr;  // counters of the double-precision decisions (3)
  DJob *djobs = nullptr;       // device job tables
  size_t djobs_cap = 0;
  DJob *hjobs = nullptr;       // pinned staging for the job tables
  cudaEvent_t staged = nullptr;
  bool staged_pending = false;
  int max_smem = 0;
  int num_sms = 0;
  int *counters = nullptr;     // persistent-kernel tile counters
  // per-kernel timing (bmnd_set_profiling)
  bool profiling = false;
  struct Mark { int kind; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
  int64_t k_launches[BMND_KERNEL_KINDS] = {0};
  double k_ms[BMND_KERNEL_KINDS] = {0};
  // tile cores chosen by bmnd_autotune, per problem key; force_core
  // overrides the planner while the tuner times a candidate
  std::map<std::string, std::vector<int>> tuned;
  const std::vector<int> *force_core = nullptr;
  // finite-count moment tables (mu, v) of the Poisson matching distances,
  // n = 0..BMND_MOMENT_NMAX, built on first use
  float2 *mom[4] = {nullptr, nullptr, nullptr, nullptr};
  // fixed-point tables of the Poisson distances for count data (PFIX_*)
  long long *pfix[4] = {nullptr, nullptr, nullptr, nullptr};
  // device copies of host arrays for bmnd_denoise_batch_host (grown on use)
  float *hio = nullptr;
  size_t hio_floats = 0;
};

namespace {

bmnd_status fail(bmnd_ctx *ctx, bmnd_status st, const char *fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define CU(call)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return fail(ctx, BMND_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

// Orthonormal DCT-II entries, computed in double.
double dct_entry(int J, int k, int i) {
  double c = k == 0 ? std::sqrt(1.0 / J) : std::sqrt(2.0 / J);
  return c * std::cos(M_PI * (2.0 * i + 1.0) * k / (2.0 * J));
}

// Modified Bessel I0 by its power series (for the Kaiser window, App. A).
double bessel_i0(double x) {
  double s = 1.0, t = 1.0, q = x * x / 4.0;
  for (int k = 1; k < 400; ++k) {
    t *= q / ((double)k * k);
    s += t;
    if (t < 1e-17 * s) break;
  }
  return s;
}

double kaiser_at(int n, int i, double beta) {
  if (n == 1) return 1.0;
  double r = 2.0 * i / (n - 1) - 1.0;
  double a = 1.0 - r * r;
  return bessel_i0(beta * std::sqrt(a > 0 ? a : 0.0)) / bessel_i0(beta);
}

// bior1.5 analysis matrix T and synthesis matrix U = T^{-1} of a periodic
// axis of J = 2^m samples (row-major J x J), full depth, coefficients
// coarsest first, as products of one dense matrix per level:
// T = W_m ... W_1 and U = V_1 ... V_m, where level s acts on the leading
// l = J / 2^(s-1) entries (the current approximation) and keeps the details
// of the finer levels in place.  Level s maps x to [a | d] with
// a[i] = sum_k lo[k] x[(2i + k) mod l] and d[i] = sum_k hi[k] x[(2i + k) mod l];
// its synthesis puts slo[k] a[i] + shi[k] d[i] back at (2i + k) mod l.
// Filters (tap k): analysis lowpass (sqrt 2 / 256) x (3, -3, -22, 22, 128,
// 128, 22, -22, -3, 3) at k = -4..5 and highpass (1, -1) / sqrt 2 at
// k = 0, 1; synthesis lowpass (1, 1) / sqrt 2 at k = 0, 1 and highpass
// shi[k] = (-1)^k lo[1 - k] -- the Cohen-Daubechies-Feauveau biorthogonal
// spline pair with a box synthesis scaling function and five vanishing
// moments of the synthesis wavelet (I. Daubechies, "Ten Lectures on
// Wavelets", 1992, Sec. 8.3).
void bior15_matrices(int J, std::vector<double> &T, std::vector<double> &U) {
  static const double taps[10] = {3, -3, -22, 22, 128, 128, 22, -22, -3, 3};
  auto lo = [&](int k) { return (k < -4 || k > 5) ? 0.0 : taps[k + 4] * std::sqrt(2.0) / 256.0; };
  auto hi = [&](int k) { return k == 0 ? std::sqrt(0.5) : (k == 1 ? -std::sqrt(0.5) : 0.0); };
  auto slo = [&](int k) { return (k == 0 || k == 1) ? std::sqrt(0.5) : 0.0; };
  auto shi = [&](int k) { return ((k & 1) ? -1.0 : 1.0) * lo(1 - k); };
  auto eye = [&](std::vector<double> &A) {
    A.assign((size_t)J * J, 0.0);
    for (int i = 0; i < J; ++i) A[(size_t)i * J + i] = 1.0;
  };
  auto mul = [&](const std::vector<double> &A, const std::vector<double> &B) {
    std::vector<double> C((size_t)J * J, 0.0);
    for (int r = 0; r < J; ++r)
      for (int k = 0; k < J; ++k) {
        const double a = A[(size_t)r * J + k];
        if (a != 0.0)
          for (int c = 0; c < J; ++c) C[(size_t)r * J + c] += a * B[(size_t)k * J + c];
      }
    return C;
  };
  eye(T);
  eye(U);
  std::vector<double> W, V;
  for (int l = J; l >= 2; l /= 2) {
    eye(W);
    eye(V);
    for (int r = 0; r < l; ++r)
      for (int c = 0; c < l; ++c) W[(size_t)r * J + c] = V[(size_t)r * J + c] = 0.0;
    for (int i = 0; i < l / 2; ++i)
      for (int k = -4; k <= 5; ++k) {
        const int c = ((2 * i + k) % l + l) % l;
        W[(size_t)i * J + c] += lo(k);
        W[(size_t)(l / 2 + i) * J + c] += hi(k);
        V[(size_t)c * J + i] += slo(k);
        V[(size_t)c * J + l / 2 + i] += shi(k);
      }
    T = mul(W, T);
    U = mul(U, V);
  }
}

std::mutex g_const_mu;
bool g_const_ready[64] = {false};

// Constants of the butterfly DCT, once per device; the device must be
// current.  Returns the CUDA error of the upload.
cudaError_t init_constants_on(int device) {
  std::lock_guard<std::mutex> lk(g_const_mu);
  if (device >= 0 && device < 64 && g_const_ready[device]) return cudaSuccess;
  float sec[31], scale[12];
  for (int N = 2; N <= 32; N *= 2)
    for (int n = 0; n < N / 2; ++n) sec[N / 2 - 1 + n] = (float)(1.0 / (2.0 * std::cos(M_PI * (2.0 * n + 1.0) / (2.0 * N))));
  for (int l = 0; l <= 5; ++l) {
    double N = (double)(1 << l);
    scale[2 * l] = (float)std::sqrt(1.0 / N);
    scale[2 * l + 1] = (float)std::sqrt(2.0 / N);
  }
  cudaError_t e = upload_fast_dct_constants(sec, scale);
  if (e == cudaSuccess && device >= 0 && device < 64) g_const_ready[device] = true;
  return e;
}

bmnd_status init_constants(bmnd_ctx *ctx) {
  CU(init_constants_on(ctx->device));
  return BMND_OK;
}

// Host image of the transform tables (TAB_BYTES): the float DCT-II matrices
// of sizes 1..32 and their entrywise squares, and the double matrices at
// TAB64_OFFSET.
void fill_tables(std::vector<unsigned char> &img) {
  img.assign(TAB_BYTES, 0);
  float *t = reinterpret_cast<float *>(img.data());
  double *t64 = reinterpret_cast<double *>(img.data() + TAB64_OFFSET);
  for (int J = 1; J <= 32; ++J) {
    int off = (J - 1) * J * (2 * J - 1) / 6;
    for (int k = 0; k < J; ++k)
      for (int i = 0; i < J; ++i) {
        double v = dct_entry(J, k, i);
        t[off + k * J + i] = (float)v;
        t[GEN_TOTAL + off + k * J + i] = (float)(v * v);
        t64[off + k * J + i] = v;
      }
    if (J & (J - 1)) continue;
    std::vector<double> T, U;
    bior15_matrices(J, T, U);
    for (int e = 0; e < J * J; ++e) {
      t[TAB_BIOR + off + e] = (float)T[e];
      t[TAB_BIOR + GEN_TOTAL + off + e] = (float)U[e];
      t64[GEN_TOTAL + off + e] = T[e];
    }
  }
}

cudaEvent_t pool_event(bmnd_ctx *ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Brackets one launch with events when profiling is on.
struct ProfScope {
  bmnd_ctx *ctx;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(bmnd_ctx *c, int k, cudaStream_t s) : ctx(c), kind(k), st(s) {
    if (ctx->profiling && (a = pool_event(ctx))) cudaEventRecord(a, st);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = pool_event(ctx);
    if (!b) { ctx->event_pool.push_back(a); return; }
    cudaEventRecord(b, st);
    ctx->marks.push_back({kind, a, b});
  }
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Geometry of one array shared by both stages.
struct Plan {
  int ndim;
  int64_t shape[BMND_MAX_NDIM];
  int patch[BMND_MAX_NDIM], step[BMND_MAX_NDIM], search[BMND_MAX_NDIM];
  int D;
  int kax_of[KMAXD];     // full axis of each kernel axis
  DGeom g;               // stage-independent part filled
  SGeom s;
  int64_t nflags;
  int Mmax;
  int gtrans;            // group transform (Haar / DCT)
  int metric;            // stage-1 matching distance (BMND_METRIC_*)
  int kex;               // shared-source variance planes (0 = diagonal)
  int spatial;           // stage-1 spatial transform (BMND_SPATIAL_*)
  int minb;              // CTAs per SM asked of the stage kernels: 0 by shared memory, 1 or 2
  int fp_candidate;
  int smem[3];           // dynamic shared bytes: stage 1, stage 2, +eta region
  // scratch offsets (bytes, relative to the job's block)
  size_t o_flags, o_refs, o_rcount, o_partial, o_pilot, o_eta, o_groups, o_gcount, total;
  // optional synthesis cache of the first mass-conservation sweep
  bool cache;
  int smem_cached;       // dynamic shared bytes of the second sweep from the cache
  int64_t cache_refs;
  size_t o_refbase, o_pcache, o_wcache;
};


// Patch side of the specialized stage kernels for a shape: they take cubic
// patches (side jL on every axis) of the sizes instantiated with the kernels,
// with a Haar group transform and the DCT spatial transform; 0 selects the
// generic kernel of the rank.
int cube_side(int D, const int *j, int gtrans, int kex, int spatial) {
  const int jL = j[D - 1];
  if (gtrans != BMND_GROUP_HAAR || spatial != BMND_SPATIAL_DCT) return 0;
  // the register filter (patches of <= 32 entries) takes at most 4
  // shared-source planes
  int P = 1;
  for (int a = 0; a < D; ++a) P *= j[a];
  if (kex > 4 && P <= 32) return 0;
  for (int a = 0; a < D; ++a)
    if (j[a] != jL) return 0;
  if ((D == 1 && (jL == 32 || jL == 16)) || (D == 2 && (jL == 8 || jL == 4)) || (D == 3 && jL == 4)) return jL;
  return 0;
}

// Dynamic shared memory of a stage launch; cached: second mass-conservation
// sweep from the synthesis cache (y and eta staged, one group buffer).
int stage_smem(const DGeom &g, int M, int nreg, bool cached = false, bool st1 = false) {
  if (cached) nreg = 2;
  else if (g.lean) nreg = 1;  // only the matching guide is staged
  size_t b = al16(sizeof(DJob));
  b = al16(b + (size_t)g.P * 12 + (size_t)g.rows * 4 + KMAXD * 4 + (g.fp ? (size_t)g.P * 4 : 0) +
           (size_t)g.fp * 4 + (g.kex ? (size_t)g.P * 4 : 0));
  b = al16(b + (g.lean ? (size_t)g.P * 8 : 0));
  size_t mats = 0;
  for (int a = 0; a < g.D; ++a) mats += (size_t)mat_block(g.j[a]) * 4;
  b = al16(b + mats);
  b = al16(b + (g.bsm && st1 && !cached ? (size_t)(g.region + RPAD) * 4 : 0));
  b = al16(b + (size_t)nreg * (g.region + RPAD) * 4);
  b = al16(b + (size_t)g.region * 8);
  b += (size_t)NW * (cached ? warp_bytes(M, g.MS, g.fp, 0, 1) : warp_bytes(M, g.MS, g.fp, g.lean));
  return (int)b;
}

// Adds the synthesis cache of the first mass-conservation sweep to a plan's
// scratch: per reference (at most one per patch origin, and at most
// passes x slots of the schedule) the M x P synthesized entries and M
// weights, plus the per-tile reference offsets.  The second sweep then
// re-aggregates without filtering again.
void add_mc_cache(Plan &pl) {
  if (pl.cache) return;
  pl.cache_refs = std::min<int64_t>(pl.nflags, (int64_t)pl.s.passes * pl.s.nslots);
  pl.o_refbase = pl.total;
  size_t o = pl.total;
  o = al256(o + (size_t)pl.g.ntiles * 4);
  pl.o_pcache = o;
  o = al256(o + (size_t)pl.cache_refs * pl.Mmax * pl.g.P * 4);
  pl.o_wcache = o;
  o = al256(o + (size_t)pl.cache_refs * pl.Mmax * 4);
  pl.total = o;
  pl.cache = true;
  pl.smem_cached = stage_smem(pl.g, pl.Mmax, 2, true);
}

void drop_mc_cache(Plan &pl) {
  if (!pl.cache) return;
  pl.total = pl.o_refbase;
  pl.cache = false;
}

void set_tiles(DGeom &g, const int *C) {
  g.ntiles = 1;
  g.cap = 1;
  g.region = 1;
  for (int d = 0; d < g.D; ++d) {
    g.C[d] = C[d];
    g.NT[d] = (int)((g.ell[d] + 1 + C[d] - 1) / C[d]);
    g.RG[d] = C[d] + 2 * g.rad[d] + g.j[d] - 1;
    g.RGP[d] = (d == g.D - 1 && g.D >= 2) ? (g.RG[d] | 1) : g.RG[d];
    g.ntiles *= g.NT[d];
    g.cap *= C[d];
    g.region *= g.RGP[d];
  }
  int s = 1;
  for (int d = g.D - 1; d >= 0; --d) { g.rst[d] = s; s *= g.RGP[d]; }
}

// Key of a problem for the tile tuner: everything the tiling depends on
// (shape, patch, step, search, group sizes, stages, mass conservation and
// the profile), not the noise level.
std::string tune_key(int ndim, const int64_t *shape, const int *patch, const int *step, const int *search,
                     const int *group_size, int stages, int mass_conserve, const bmnd_params &pr) {
  std::string k;
  char b[96];
  for (int d = 0; d < ndim; ++d) {
    snprintf(b, sizeof(b), "%lld/%d/%d/%d;", (long long)shape[d], patch[d], step[d], search[d]);
    k += b;
  }
  snprintf(b, sizeof(b), "g%d,%d s%d m%d t%d sc%d p%d w%d,%d d%d", group_size[0], stages == 2 ? group_size[1] : 0,
           stages, mass_conserve, pr.group_transform, pr.schedule, pr.passes, pr.weight_model, pr.weight_scope,
           pr.match_metric + 16 * pr.cov_planes + 1024 * pr.spatial_transform);
  k += b;
  return k;
}

// Per-entry contribution phi_m(r, c) of a Poisson matching distance
// (Eq. varphi), double precision: deviance (0 log 0 = 0), Pearson and half
// the squared Anscombe difference; a zero pooled count contributes 0.
double contribution(int metric, double r, double c) {
  const double n = r + c;
  if (metric == BMND_METRIC_DEVIANCE) {
    if (n <= 0) return 0.0;
    return 2.0 * ((r > 0 ? r * std::log(2.0 * r / n) : 0.0) + (c > 0 ? c * std::log(2.0 * c / n) : 0.0));
  }
  if (metric == BMND_METRIC_PEARSON) return n > 0 ? (r - c) * (r - c) / n : 0.0;
  const double d = 2.0 * std::sqrt(c + 0.375) - 2.0 * std::sqrt(r + 0.375);
  return 0.5 * d * d;
}

// Finite-count null moments (Prop. "Universal finite-count moments") for
// n = 0..count-1.  The Binomial(n, 1/2) weights of row n come from row n-1 by
// Pascal's rule, w_n(x) = (w_{n-1}(x) + w_{n-1}(x-1)) / 2.  n = 0 has the
// single allocation (0, 0); at n = 1 both allocations contribute equally, so
// v = 0 exactly.  A variance that rounding makes negative becomes 0.
void moment_table64(int metric, int count, std::vector<double2> &out) {
  out.assign(count, make_double2(0.0, 0.0));
  std::vector<double> w(count + 1, 0.0);
  w[0] = 1.0;
  for (int n = 1; n < count; ++n) {
    for (int x = n; x >= 1; --x) w[x] = 0.5 * (w[x] + w[x - 1]);
    w[0] *= 0.5;
    if (n == 1) {
      out[1] = make_double2(contribution(metric, 1.0, 0.0), 0.0);
      continue;
    }
    double m1 = 0, m2 = 0;
    for (int x = 0; x <= n; ++x) {
      if (w[x] == 0.0) continue;
      const double f = contribution(metric, (double)x, (double)(n - x));
      m1 += w[x] * f;
      m2 += w[x] * f * f;
    }
    out[n] = make_double2(m1, std::max(m2 - m1 * m1, 0.0));
  }
}

void moment_table(int metric, int count, std::vector<float2> &out) {
  std::vector<double2> m;
  moment_table64(metric, count, m);
  out.resize(count);
  for (int n = 0; n < count; ++n) out[n] = make_float2((float)m[n].x, (float)m[n].y);
}

// Fixed-point tables of one Poisson distance (layout PFIX_* of the kernel
// header): the per-entry contributions of Eqs. (deviance), (pearson),
// (anscombe-distance) at integer counts in closed form, and the moments.
void fixed_tables(int metric, std::vector<long long> &t) {
  t.assign(PFIX_TOTAL, 0);
  const double two32 = 4294967296.0;
  for (int k = 0; k <= PFIX_K; ++k) {
    const double K = (double)k;
    if (metric == BMND_METRIC_DEVIANCE) {
      t[PFIX_A + k] = k > 0 ? std::llround(K * std::log(2.0 * K) * two32) : 0;
      t[PFIX_B + k] = k > 1 ? std::llround(K * std::log(K) * two32) : 0;
    } else if (metric == BMND_METRIC_PEARSON) {
      t[PFIX_A + k] = k > 1 ? (long long)(((unsigned __int128)1 << 64) / (unsigned)k)
                            : (k == 1 ? (long long)~0ull : 0);
    } else {
      t[PFIX_A + k] = std::llround(2.0 * std::sqrt(K + 0.375) * 17592186044416.0);  // 2^44
    }
  }
  std::vector<double2> m;
  moment_table64(metric, BMND_MOMENT_NMAX + 1, m);
  for (int n = 0; n <= BMND_MOMENT_NMAX; ++n) {
    t[PFIX_MU + n] = std::llround(m[n].x * two32);
    t[PFIX_V + n] = std::llround(m[n].y * two32);
  }
}

bmnd_status ensure_moments(bmnd_ctx *ctx, int metric) {
  if (ctx->mom[metric]) return BMND_OK;
  std::vector<float2> h;
  moment_table(metric, BMND_MOMENT_NMAX + 1, h);
  float2 *d = nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BMND_ENOMEM, "cudaMalloc of the moment table failed");
  }
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d);
    return fail(ctx, BMND_ECUDA, "upload of the moment table failed");
  }
  ctx->mom[metric] = d;
  std::vector<long long> t;
  fixed_tables(metric, t);
  long long *dt = nullptr;
  if (cudaMalloc(&dt, t.size() * sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BMND_ENOMEM, "cudaMalloc of the fixed-point tables failed");
  }
  if (cudaMemcpy(dt, t.data(), t.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dt);
    return fail(ctx, BMND_ECUDA, "upload of the fixed-point tables failed");
  }
  ctx->pfix[metric] = dt;
  return BMND_OK;
}

bmnd_status make_plan(bmnd_ctx *ctx, int ndim, const int64_t *shape, const int *patch, const int *step,
                      const int *search, const int *group_size, int stages, int mass_conserve,
                      const bmnd_params &pr, Plan &pl) {
  if (ndim < 1 || ndim > BMND_MAX_NDIM) return fail(ctx, BMND_EINVAL, "ndim %d not in [1, %d]", ndim, BMND_MAX_NDIM);
  if (!shape || !patch || !step || !search) return fail(ctx, BMND_EINVAL, "null shape/patch/step/search");
  if (stages != 1 && stages != 2) return fail(ctx, BMND_EINVAL, "stages must be 1 or 2");
  pl.ndim = ndim;
  int64_t N = 1;
  for (int d = 0; d < ndim; ++d) {
    if (shape[d] < 1) return fail(ctx, BMND_EINVAL, "shape[%d] = %lld < 1", d, (long long)shape[d]);
    if (patch[d] < 1 || patch[d] > shape[d]) return fail(ctx, BMND_EINVAL, "patch[%d] = %d not in [1, shape]", d, patch[d]);
    if (patch[d] > JMAX) return fail(ctx, BMND_EINVAL, "patch[%d] = %d exceeds %d", d, patch[d], JMAX);
    if (step[d] < 1 || step[d] > patch[d]) return fail(ctx, BMND_EINVAL, "step[%d] = %d not in [1, patch]", d, step[d]);
    if (search[d] < 1 || search[d] % 2 == 0) return fail(ctx, BMND_EINVAL, "search[%d] = %d must be odd and >= 1", d, search[d]);
    pl.shape[d] = shape[d];
    pl.patch[d] = patch[d];
    pl.step[d] = step[d];
    pl.search[d] = search[d];
    N *= shape[d];
  }
  if (N >= ((int64_t)1 << 40)) return fail(ctx, BMND_EINVAL, "array too large");
  for (int s = 0; s < stages; ++s) {
    int M = group_size[s];
    if (M < 1 || M > MMAX) return fail(ctx, BMND_EINVAL, "group_size[%d] = %d not in [1, %d]", s, M, MMAX);
    if (pr.group_transform == BMND_GROUP_HAAR && (M & (M - 1)))
      return fail(ctx, BMND_EINVAL, "group_size[%d] = %d is not a power of two (Haar)", s, M);
  }
  if (pr.min_group < 1) return fail(ctx, BMND_EINVAL, "min_group < 1");
  if (pr.passes < 1) return fail(ctx, BMND_EINVAL, "passes < 1");
  if (pr.schedule < 0 || pr.schedule > 3) return fail(ctx, BMND_EINVAL, "unknown schedule");
  if (pr.group_transform < 0 || pr.group_transform > 1) return fail(ctx, BMND_EINVAL, "unknown group transform");
  if (pr.weight_model < 0 || pr.weight_model > 2 || pr.weight_scope < 0 || pr.weight_scope > 1)
    return fail(ctx, BMND_EINVAL, "unknown weight model/scope");
  if (pr.power_mode < 0 || pr.power_mode > 2) return fail(ctx, BMND_EINVAL, "unknown power mode");
  if (pr.ht_rule < 0 || pr.ht_rule > 1) return fail(ctx, BMND_EINVAL, "unknown thresholding rule");
  if (pr.weight_domain < 0 || pr.weight_domain > 1) return fail(ctx, BMND_EINVAL, "unknown weight domain");
  if (pr.cov_planes < 0 || pr.cov_planes > MMAX) return fail(ctx, BMND_EINVAL, "cov_planes not in [0, %d]", MMAX);
  if (pr.spatial_transform != BMND_SPATIAL_DCT && pr.spatial_transform != BMND_SPATIAL_BIOR15)
    return fail(ctx, BMND_EINVAL, "unknown spatial transform");
  if (pr.spatial_transform == BMND_SPATIAL_BIOR15)
    for (int d = 0; d < ndim; ++d)
      if (patch[d] & (patch[d] - 1))
        return fail(ctx, BMND_EINVAL, "bior1.5 needs power-of-two patch sides (patch[%d] = %d)", d, patch[d]);
  if (pr.match_metric < 0 || pr.match_metric > 3) return fail(ctx, BMND_EINVAL, "unknown matching distance");
  if (pr.match_policy < 0 || pr.match_policy > 2) return fail(ctx, BMND_EINVAL, "unknown matching policy");
  if (pr.match_metric != BMND_METRIC_SSD && (!(pr.match_t >= 0) || !(pr.beta_s >= 0) || !(pr.kappa_s > 0)))
    return fail(ctx, BMND_EINVAL, "match_t and beta_s must be >= 0 and kappa_s > 0");
  if (!(pr.shift_density >= 0) || !(pr.s_v >= 0) || !(pr.lambda_ht >= 0))
    return fail(ctx, BMND_EINVAL, "negative shift_density, s_v or lambda_ht");
  // kernel axes: those with length > 1 (at least one)
  int D = 0;
  for (int d = 0; d < ndim; ++d)
    if (shape[d] > 1) {
      if (D == KMAXD) return fail(ctx, BMND_EUNSUPPORTED, "more than %d axes of length > 1", KMAXD);
      pl.kax_of[D++] = d;
    }
  if (D == 0) pl.kax_of[D++] = ndim - 1;
  pl.D = D;
  DGeom &g = pl.g;
  memset(&g, 0, sizeof(g));
  g.D = D;
  g.N = N;
  g.P = 1;
  for (int a = 0; a < D; ++a) {
    int d = pl.kax_of[a];
    g.L[a] = shape[d];
    g.j[a] = patch[d];
    g.rad[a] = (search[d] - 1) / 2;
    g.ell[a] = shape[d] - patch[d];
    g.P *= patch[d];
    for (int i = 0; i < JMAX; ++i) g.kaiser[a][i] = i < patch[d] ? (float)kaiser_at(patch[d], i, pr.kaiser_beta) : 0.f;
  }
  {
    int64_t s = 1;
    for (int a = D - 1; a >= 0; --a) { g.st[a] = s; s *= g.L[a]; }
  }
  g.jL = g.j[D - 1];
  g.rows = g.P / g.jL;
  // with three or more axes the halo of a tile (2 rad + j - 1 per axis)
  // dominates its region: read y and eta from global memory and spend the
  // shared memory on larger tiles
  g.lean = D >= 3 ? 1 : 0;
  pl.gtrans = pr.group_transform;
  pl.metric = pr.match_metric;
  pl.kex = pr.cov_planes;
  pl.spatial = pr.spatial_transform;
  pl.minb = 0;
  g.kex = pr.cov_planes;  // the shared-memory plan holds the coordinate table
  // patch-sum map for the stage-1 noise bias: specialized kernels with one
  // or two axes (with three, the lean tiles spend the memory on cores)
  g.bsm = (D <= 2 && cube_side(D, g.j, pl.gtrans, pl.kex, pl.spatial)) ? 1 : 0;
  g.dct64 = ctx->tab64;
  g.diag = ctx->diag;
  if (pl.metric != BMND_METRIC_SSD) {
    bmnd_status rc = ensure_moments(ctx, pl.metric);
    if (rc != BMND_OK) return rc;
    g.mom = ctx->mom[pl.metric];
    g.pfix = ctx->pfix[pl.metric];
  }
  if (cube_side(D, g.j, pl.gtrans, pl.kex, pl.spatial) && g.P <= 32) {
    // specialized kernels with members in registers: unpadded rows, odd
    // member stride (whole members and whole entry columns are read)
    g.LS = g.jL;
    g.MS = g.P | 1;
  } else {
    // group-buffer line stride: odd (bank-conflict free lines), except in
    // lean mode with rows of a multiple of 4 floats, where the unpadded
    // layout keeps stride-1 lines float4-aligned and saves a fifth of the
    // warp buffers
    g.LS = (g.lean && g.jL % 4 == 0) ? g.jL : g.jL + (g.jL % 2 == 0 ? 1 : 0);
    g.MS = g.rows * g.LS;
  }
  // private group footprint for the accumulation when it is small
  {
    int64_t fp = 1;
    for (int a = 0; a < D; ++a) {
      g.FW[a] = 2 * g.rad[a] + g.j[a];
      fp *= g.FW[a];
    }
    g.fp = 0;
    pl.fp_candidate = fp <= 1024 ? (int)fp : 0;
  }
  pl.Mmax = group_size[0];
  if (stages == 2) pl.Mmax = std::max(pl.Mmax, group_size[1]);
  // tile geometry: large cores within the shared-memory budget, enough tiles
  static const int target[KMAXD + 1] = {0, 64, 32, 8, 4, 3, 2};
  static const int minc[KMAXD + 1] = {0, 32, 8, 4, 2, 2, 1};
  int C[KMAXD];
  for (int a = 0; a < D; ++a) C[a] = (int)std::min<int64_t>(target[D], g.ell[a] + 1);
  int nreg_max = (stages == 2 ? 2 : 1) + (mass_conserve ? 1 : 0);
  // shared memory of the largest launch of the plan: stage 1 (with its
  // patch-sum map), stage 2 and the mass-conservation sweep
  auto plan_smem = [&](const DGeom &gg) {
    return std::max(stage_smem(gg, pl.Mmax, nreg_max), stage_smem(gg, group_size[0], 1, false, true));
  };
  if (D >= 3) {
    // every core shape up to the target: the smallest staged region per core
    // location, discounted while there are fewer than 2 tiles per SM
    int best[KMAXD] = {0}, lim[KMAXD];
    double best_cost = 0.0;
    for (int a = 0; a < D; ++a) { lim[a] = C[a]; C[a] = 1; }
    for (;;) {
      set_tiles(g, C);
      if (plan_smem(g) <= ctx->max_smem) {
        const double cost = (double)g.region / (double)g.cap / (double)std::min<int64_t>(g.ntiles, 2 * 148);
        if (best[0] == 0 || cost < best_cost) {
          best_cost = cost;
          for (int a = 0; a < D; ++a) best[a] = C[a];
        }
      }
      int a = D - 1;
      while (a >= 0 && C[a] == lim[a]) C[a--] = 1;
      if (a < 0) break;
      ++C[a];
    }
    if (best[0] == 0) return fail(ctx, BMND_EUNSUPPORTED, "patch/group too large for shared memory (P=%d, M=%d)", g.P, pl.Mmax);
    for (int a = 0; a < D; ++a) C[a] = best[a];
    set_tiles(g, C);
  }
  // one or two axes: halve the largest core side until the tile fits and
  // there are 2 tiles per SM (or the cores reach their minimum)
  while (D < 3) {
    set_tiles(g, C);
    bool fits = plan_smem(g) <= ctx->max_smem;
    int big = 0;
    for (int a = 1; a < D; ++a) if (C[a] > C[big]) big = a;
    if (fits && (g.ntiles >= 2 * 148 || C[big] < 2 * minc[D])) break;
    if (C[big] == 1) {
      if (!fits) return fail(ctx, BMND_EUNSUPPORTED, "patch/group too large for shared memory (P=%d, M=%d)", g.P, pl.Mmax);
      break;
    }
    C[big] = (C[big] + 1) / 2;
  }
  // a core chosen by bmnd_autotune for this problem (or forced while the
  // tuner times it), if it fits
  {
    const std::vector<int> *core = ctx->force_core;
    if (!core) {
      auto it = ctx->tuned.find(tune_key(ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr));
      if (it != ctx->tuned.end()) core = &it->second;
    }
    if (core && ((int)core->size() == D || (int)core->size() == D + 1)) {
      if ((int)core->size() == D + 1) pl.minb = (*core)[D];
      int T[KMAXD];
      bool ok = true;
      for (int a = 0; a < D; ++a) {
        T[a] = (*core)[a];
        ok = ok && T[a] >= 1 && T[a] <= g.ell[a] + 1;
      }
      if (ok) {
        set_tiles(g, T);
        if (plan_smem(g) <= ctx->max_smem) {
          for (int a = 0; a < D; ++a) C[a] = T[a];
        } else {
          set_tiles(g, C);
        }
      }
    }
  }
  // enable the private footprint if it costs no resident CTA per SM
  if (pl.fp_candidate) {
    const int per_sm = 233472;  // shared memory per SM
    int without = plan_smem(g);
    g.fp = pl.fp_candidate;
    int with = plan_smem(g);
    int b0 = std::min(2, per_sm / std::max(without, 1)), b1 = std::min(2, per_sm / std::max(with, 1));
    if (with > ctx->max_smem || b1 < b0) g.fp = 0;
  }
  pl.smem[0] = stage_smem(g, group_size[0], 1, false, true);
  pl.smem[1] = stages == 2 ? stage_smem(g, group_size[1], 2) : 0;
  pl.smem[2] = stage_smem(g, pl.Mmax, nreg_max);
  // schedule geometry on the full shape
  SGeom &s = pl.s;
  memset(&s, 0, sizeof(s));
  s.ndim = ndim;
  s.schedule = pr.schedule;
  s.passes = pr.schedule == BMND_SCHEDULE_OFF ? 1 : pr.passes;
  s.rho = pr.shift_density;
  s.D = D;
  s.nslots = 1;
  for (int d = 0; d < ndim; ++d) {
    s.j[d] = patch[d];
    s.h[d] = step[d];
    s.ell[d] = shape[d] - patch[d];
    s.Z[d] = (s.ell[d] + step[d] - 1) / step[d] + 1;
    s.nslots *= s.Z[d];
    s.kax[d] = -1;
  }
  for (int a = 0; a < D; ++a) s.kax[pl.kax_of[a]] = a;
  pl.nflags = 1;
  for (int a = D - 1; a >= 0; --a) { s.fst[a] = pl.nflags; pl.nflags *= g.ell[a] + 1; }
  // scratch
  size_t o = 0;
  pl.o_flags = o; o = al256(o + (size_t)pl.nflags);
  pl.o_refs = o; o = al256(o + (size_t)g.ntiles * g.cap * 4);
  pl.o_rcount = o; o = al256(o + (size_t)g.ntiles * 4);
  pl.o_partial = o; o = al256(o + (size_t)g.ntiles * g.region * 8);
  pl.o_pilot = o; o = al256(o + (stages == 2 ? (size_t)N * 4 : 0));
  pl.o_eta = o; o = al256(o + (mass_conserve ? (size_t)N * 4 : 0));
  pl.o_groups = o; o = al256(o + (size_t)g.ntiles * g.cap * pl.Mmax * 4);
  pl.o_gcount = o; o = al256(o + (size_t)g.ntiles * g.cap * 4);
  pl.total = o;
  pl.cache = false;
  pl.cache_refs = 0;
  pl.o_refbase = pl.o_pcache = pl.o_wcache = 0;
  return BMND_OK;
}

void fill_stage(DGeom &g, int stage, int M, const bmnd_noise &nz, const bmnd_params &pr) {
  g.stage = stage;
  g.M = M;
  g.min_group = pr.min_group;
  g.gtrans = pr.group_transform;
  g.wmodel = pr.weight_model;
  g.wscope = pr.weight_scope;
  g.poisson = nz.kind == BMND_NOISE_POISSON;
  double gamma = stage == 1 ? pr.gamma_ht : pr.gamma_wie;
  g.gamma = (float)gamma;
  // Poisson matching distances in stage 1 only (App. B: the Wiener stage
  // matches the pilot by SSD with a fixed threshold)
  g.metric = stage == 1 ? pr.match_metric : BMND_METRIC_SSD;
  g.policy = pr.match_policy;
  g.bias_on = g.poisson && gamma > 0 && g.metric == BMND_METRIC_SSD;
  double tau = stage == 1 ? pr.tau_ht : pr.tau_wie;
  if (tau <= 0) tau = (stage == 1 ? 3000.0 : 400.0) * g.P / (255.0 * 255.0);
  g.tau = (float)tau;
  if (g.metric != BMND_METRIC_SSD) {
    // thresholds in sum units, P d_m (fixed: tau_ht or the high-count null
    // 1 + t sqrt(2 / P); standardized: t; reference: per reference patch)
    if (g.policy == BMND_POLICY_FIXED) {
      double tf = pr.tau_ht > 0 ? pr.tau_ht : 1.0 + pr.match_t * std::sqrt(2.0 / g.P);
      g.tau = (float)(tf * g.P);
    } else if (g.policy == BMND_POLICY_STANDARDIZED) {
      g.tau = (float)pr.match_t;
    }
    g.mt = (float)pr.match_t;
    g.beta_p = (float)(pr.beta_s * g.P);
    g.kappa = (float)pr.kappa_s;
    g.mt64 = pr.match_t;
    g.beta_p64 = pr.beta_s * (double)g.P;
    g.kappa64 = pr.kappa_s;
    g.inv_sp = (float)(1.0 / nz.poisson_scale);
  }
  g.lambda = (float)pr.lambda_ht;
  g.soft = stage == 1 && pr.ht_rule == BMND_HT_SOFT;
  g.wdomain = pr.weight_domain;
  g.kex = pr.cov_planes;
  g.s_v = (float)pr.s_v;
  g.a_power = pr.power_mode == 0 ? 0.f : (pr.power_mode == 1 ? 1.f : (float)pr.s_v);
  g.s_p = (float)(g.poisson ? nz.poisson_scale : 1.0);
  g.var_g = (float)(g.poisson ? 0.0 : nz.sigma * nz.sigma);
  // double-precision decisions: the scalars as the definitions have them
  // (the Gaussian bias as 2 P sigma^2, evaluated left to right)
  g.s_p64 = g.poisson ? nz.poisson_scale : 1.0;
  g.gamma64 = g.metric == BMND_METRIC_SSD ? gamma : 0.0;
  g.gbias64 = g.poisson ? 0.0 : 2.0 * (double)g.P * nz.sigma * nz.sigma;
  g.tau64 = tau;
  if (g.metric != BMND_METRIC_SSD) {
    if (g.policy == BMND_POLICY_FIXED) {
      const double tf = pr.tau_ht > 0 ? pr.tau_ht : 1.0 + pr.match_t * std::sqrt(2.0 / g.P);
      g.tau64 = tf * g.P;
    } else if (g.policy == BMND_POLICY_STANDARDIZED) {
      g.tau64 = pr.match_t;
    }
  }
  g.lambda64 = pr.lambda_ht;
  g.var64 = g.poisson ? 0.0 : nz.sigma * nz.sigma;
  // |s32 - s| <= (P + 6) 2^-24 (ssd + gamma B) for the FP32 score (one
  // rounding per entry in the SSD and the bias sums, a few in the
  // combination), with margin
  g.ku = (float)((g.P + 8) * std::ldexp(1.0, -24) * 1.05);
  // Poisson distances on count data: exact integer sums, so a float key is
  // off by its own rounding only (the standardized one by a few roundings)
  if (g.metric != BMND_METRIC_SSD) g.ku = (float)std::ldexp(1.0, g.policy == BMND_POLICY_STANDARDIZED ? -20 : -22);
  // spatial transform: bior1.5 in stage 1 when selected (App. A), else the
  // DCT.  ht_t2 bounds the squared entries of the spatial transform (2 / J
  // per DCT axis); the dense non-orthonormal bior1.5 path gets a 4x wider
  // FP32 hard-threshold band.  Windowed synthesis metric factor of axis a
  // (Def. "Windowed synthesis metrics"): sum_p S(p, q)^2 kaiser(p)^2 over
  // the synthesis S of the axis (S = DCT^T).
  g.spatial = stage == 1 && pr.spatial_transform == BMND_SPATIAL_BIOR15 ? 1 : 0;
  g.sp64 = g.dct64 ? g.dct64 + (g.spatial ? GEN_TOTAL : 0) : nullptr;
  g.ht_band = g.spatial ? 4.f : 1.f;
  double t2 = 1.0;
  for (int a = 0; a < g.D; ++a) {
    const int J = g.j[a];
    std::vector<double> T, U;
    if (g.spatial) bior15_matrices(J, T, U);
    double mx = 0.0;
    for (int q = 0; q < JMAX; ++q) {
      double e = 0.0;
      if (q < J)
        for (int i = 0; i < J; ++i) {
          const double c = g.spatial ? U[(size_t)i * J + q] : dct_entry(J, q, i);
          const double k = kaiser_at(J, i, pr.kaiser_beta);
          e += c * c * k * k;
          const double f = g.spatial ? T[(size_t)q * J + i] : c;
          mx = std::max(mx, f * f);
        }
      g.wsyn[a][q] = (float)e;
    }
    t2 *= g.spatial ? mx : (J >= 2 ? 2.0 / J : 1.0);
  }
  g.ht_t2 = (float)t2;
  int ex = 0;
  const bool pow2 = g.poisson && std::frexp(nz.poisson_scale, &ex) == 0.5;
  g.exact_ok = stage == 1 && g.metric == BMND_METRIC_SSD && pow2 && gamma >= 0 && gamma <= 64 &&
               gamma == std::floor(gamma);
}

// Patch side of the specialized stage kernel for a plan (0: generic).
int kernel_jl(const Plan &pl) { return cube_side(pl.D, pl.g.j, pl.gtrans, pl.kex, pl.spatial); }

// Kernel stage of a plan's stage s: 3 selects the stage-1 kernels with a
// Poisson matching distance.
int kernel_stage(int metric, int s) { return s == 1 && metric != BMND_METRIC_SSD ? 3 : s; }

// Candidates per lane of the matching loop for the plan's stage kernel.
int pick_kb(const Plan &pl) {
  const int D = pl.D, jL = kernel_jl(pl);
  if (D == 1 && jL == 32) return 5;
  if (D == 1 && jL == 16) return 4;
  if (D == 2 && jL == 8) return 8;
  if (D == 3 && jL == 4) return 11;
  return 4;
}

bmnd_status ensure_arena(bmnd_ctx *ctx, size_t need, cudaStream_t st) {
  if (ctx->budget && need > ctx->budget)
    return fail(ctx, BMND_ENOMEM, "scratch need %zu bytes exceeds budget %zu", need, ctx->budget);
  if (need <= ctx->arena_size) return BMND_OK;
  CU(cudaStreamSynchronize(st));
  CU(cudaDeviceSynchronize());
  if (ctx->arena) CU(cudaFree(ctx->arena));
  ctx->arena = nullptr;
  ctx->arena_size = 0;
  size_t sz = need + need / 8;
  if (cudaMalloc(&ctx->arena, sz) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, BMND_ENOMEM, "cudaMalloc of %zu scratch bytes failed", sz);
  }
  ctx->arena_size = sz;
  return BMND_OK;
}

// Launch the stage kernel: tiles handed out by an atomic counter that is
// cleared first (the context's unless another is given); one CTA per resident
// slot (persistent), or one CTA per tile when tile_ctas is set, which lets the
// block scheduler place higher-priority work between tiles.  Every job of the
// launch runs the given stage (1 or 2).
bmnd_status launch_stage(bmnd_ctx *ctx, int D, int jL, int kb, int stage, const DJob *dj, int nj, int tiles,
                         int mode, int smem, cudaStream_t st, int *counter = nullptr, bool tile_ctas = false,
                         int minb_pref = 0) {
  // two CTAs per SM (a register cap of 128) when their shared memory fits,
  // else the full register file; a tuned preference of one CTA per SM wins
  int minb = 2 * (smem + 1024) <= 233472 ? 2 : 1;
  if (minb_pref == 1) minb = 1;
  stage_fn f = select_stage_kernel(D, jL, kb, minb, stage);
  CU(set_stage_smem(f, smem));
  int per_sm = 0;
  CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)f, NW * 32, smem));
  if (per_sm < 1) return fail(ctx, BMND_EUNSUPPORTED, "stage kernel does not fit on an SM (%d bytes)", smem);
  if (!counter) counter = ctx->counters;
  int grid = tile_ctas ? tiles : std::min(tiles, per_sm * ctx->num_sms);
  CU(cudaMemsetAsync(counter, 0, sizeof(int), st));
  f<<<grid, NW * 32, smem, st>>>(dj, nj, tiles, mode, ctx->tab, counter);
  CU(cudaGetLastError());
  return BMND_OK;
}

bmnd_status stage_jobs(bmnd_ctx *ctx, const std::vector<DJob> &h, cudaStream_t st) {
  size_t n = h.size();
  if (n > ctx->djobs_cap) {
    CU(cudaStreamSynchronize(st));
    if (ctx->djobs) CU(cudaFree(ctx->djobs));
    if (ctx->hjobs) CU(cudaFreeHost(ctx->hjobs));
    ctx->djobs = nullptr;
    ctx->hjobs = nullptr;
    size_t cap = std::max<size_t>(n, 64);
    CU(cudaMalloc(&ctx->djobs, cap * sizeof(DJob)));
    CU(cudaMallocHost(&ctx->hjobs, cap * sizeof(DJob)));
    ctx->djobs_cap = cap;
    ctx->staged_pending = false;
  }
  if (ctx->staged_pending) CU(cudaEventSynchronize(ctx->staged));
  memcpy(ctx->hjobs, h.data(), n * sizeof(DJob));
  CU(cudaMemcpyAsync(ctx->djobs, ctx->hjobs, n * sizeof(DJob), cudaMemcpyHostToDevice, st));
  CU(cudaEventRecord(ctx->staged, st));
  ctx->staged_pending = true;
  return BMND_OK;
}

struct JobIO {
  const float *y;
  float *out;
  bmnd_noise noise;
  int group_size[2];
  int stages;
  int mass_conserve;
};

bmnd_status check_noise(bmnd_ctx *ctx, const bmnd_noise &nz, const bmnd_params *pr = nullptr) {
  if (nz.kind == BMND_NOISE_GAUSSIAN) {
    if (!(nz.sigma >= 0)) return fail(ctx, BMND_EINVAL, "Gaussian sigma must be >= 0");
  } else if (nz.kind == BMND_NOISE_POISSON) {
    if (!(nz.poisson_scale > 0)) return fail(ctx, BMND_EINVAL, "Poisson scale must be > 0");
  } else {
    return fail(ctx, BMND_EINVAL, "unknown noise kind %d", nz.kind);
  }
  // the Poisson matching distances are defined on raw counts y / s_P
  if (pr && pr->match_metric != BMND_METRIC_SSD && nz.kind != BMND_NOISE_POISSON)
    return fail(ctx, BMND_EINVAL, "Poisson matching distances need the scaled-Poisson noise model");
  if (pr && pr->cov_planes > 0 && nz.kind != BMND_NOISE_POISSON)
    return fail(ctx, BMND_EINVAL, "the shared-source variance model needs the scaled-Poisson noise model");
  return BMND_OK;
}

// Job tables of several arrays laid out from scratch base A (job i at
// A + base[i]): h = [stage 1 | stage 2] descriptors, plus what the launches
// need.  first_stage / last_stage select a sub-range (bmnd_stage runs one
// stage with an external pilot).
struct JobTables {
  std::vector<DJob> h;
  int nj = 0, D = 0, tiles = 0;
  int64_t vox = 0;
  int smax[2] = {0, 0}, smax2[2] = {0, 0};
  bool any_mc[2] = {false, false};
  int kjL = 0, kkb = 4;
  int kmetric = 0;        // stage-1 matching distance shared by the jobs
  int kminb = 0;          // CTAs per SM asked of the stage kernels (0: by shared memory)
};

void build_tables(const std::vector<Plan> &plans, const std::vector<JobIO> &io, const bmnd_params &pr,
                  int first_stage, int last_stage, const float *ext_pilot, char *A, const std::vector<size_t> &base,
                  JobTables &t) {
  const int nj = (int)plans.size();
  t.nj = nj;
  t.D = plans[0].D;
  t.h.assign(2 * nj, DJob());
  for (int i = 0; i < nj; ++i) {
    const Plan &pl = plans[i];
    char *B = A + base[i];
    for (int s = 1; s <= 2; ++s) {
      DJob &J = t.h[(s - 1) * nj + i];
      memset(&J, 0, sizeof(J));
      J.g = pl.g;
      int M = io[i].group_size[s - 1];
      fill_stage(J.g, s, M, io[i].noise, pr);
      bool mc = (io[i].mass_conserve >> (s - 1)) & 1;
      bool last = s == io[i].stages || s == last_stage;
      float *pilot = (float *)(B + pl.o_pilot);
      if (s == 1 && first_stage == 2) continue;
      J.y = io[i].y;
      J.guide = s == 1 ? io[i].y : (ext_pilot ? ext_pilot : pilot);
      J.out = last ? io[i].out : pilot;
      J.eta = mc ? (float *)(B + pl.o_eta) : nullptr;
      J.partial = (float2 *)(B + pl.o_partial);
      J.ref_local = (const int *)(B + pl.o_refs);
      J.ref_count = (const int *)(B + pl.o_rcount);
      J.groups = mc ? (int *)(B + pl.o_groups) : nullptr;
      J.gcount = mc ? (int *)(B + pl.o_gcount) : nullptr;
      if (mc && pl.cache) {
        J.pcache = (float *)(B + pl.o_pcache);
        J.wcache = (float *)(B + pl.o_wcache);
        J.ref_base = (const int *)(B + pl.o_refbase);
        J.pcache_refs = pl.cache_refs;
      }
      J.tile_base = t.tiles;
      J.vox_base = t.vox;
      if (mc) t.any_mc[s - 1] = true;
      t.smax[s - 1] = std::max(t.smax[s - 1], mc ? std::max(pl.smem[s - 1], pl.smem[2]) : pl.smem[s - 1]);
      if (mc)
        t.smax2[s - 1] =
            std::max(t.smax2[s - 1], pl.cache ? pl.smem_cached : std::max(pl.smem[s - 1], pl.smem[2]));
    }
    t.tiles += pl.g.ntiles;
    t.vox += pl.g.N;
  }
  t.kjL = kernel_jl(plans[0]);
  t.kkb = pick_kb(plans[0]);
  t.kmetric = plans[0].metric;
  t.kminb = plans[0].minb;
  for (int i = 1; i < nj; ++i)
    if (kernel_jl(plans[i]) != t.kjL) { t.kjL = 0; t.kkb = 4; }
}

// The launches of both requested stages, with the job tables already on the
// device at dtab and tile counter `counter`: schedules, stage kernels,
// reductions (and the second mass-conservation sweeps).  Only stream work:
// it can be recorded into a CUDA graph.
bmnd_status record_launches(bmnd_ctx *ctx, const std::vector<Plan> &plans, const JobTables &t, char *A,
                            const std::vector<size_t> &base, int first_stage, int last_stage, DJob *dtab,
                            int *counter, cudaStream_t st) {
  const int nj = t.nj, D = t.D;
  // schedule of every job (shared by both stages)
  for (int i = 0; i < nj; ++i) {
    const Plan &pl = plans[i];
    char *B = A + base[i];
    CU(cudaMemsetAsync(B + pl.o_flags, 0, (size_t)pl.nflags, st));
    ProfScope ps(ctx, BMND_KERNEL_SCHEDULE, st);
    launch_sched(pl.s, (unsigned char *)(B + pl.o_flags), dtab + (first_stage == 2 ? nj : 0) + i,
                 pl.g.ntiles, (int *)(B + pl.o_refs), (int *)(B + pl.o_rcount), st);
    if (pl.cache) launch_ref_base((const int *)(B + pl.o_rcount), pl.g.ntiles, (int *)(B + pl.o_refbase), st);
  }
  CU(cudaGetLastError());
  const int rgrid = (int)std::min<int64_t>((t.vox + 255) / 256, 148 * 32);
  for (int s = first_stage; s <= last_stage; ++s) {
    const DJob *dj = dtab + (s - 1) * nj;
    bmnd_status rc;
    {
      ProfScope ps(ctx, s == 1 ? BMND_KERNEL_STAGE1 : BMND_KERNEL_STAGE2, st);
      rc = launch_stage(ctx, D, t.kjL, t.kkb, kernel_stage(t.kmetric, s), dj, nj, t.tiles, 0, t.smax[s - 1], st,
                        counter, false, t.kminb);
    }
    if (rc != BMND_OK) return rc;
    {
      ProfScope ps(ctx, BMND_KERNEL_REDUCE, st);
      launch_reduce(D, dj, nj, t.vox, t.any_mc[s - 1] ? 1 : 0, rgrid, st);
    }
    CU(cudaGetLastError());
    if (t.any_mc[s - 1]) {
      {
        ProfScope ps(ctx, BMND_KERNEL_MC_SWEEP, st);
        rc = launch_stage(ctx, D, t.kjL, t.kkb, kernel_stage(t.kmetric, s), dj, nj, t.tiles, 2, t.smax2[s - 1], st,
                          counter, false, t.kminb);
      }
      if (rc != BMND_OK) return rc;
      {
        ProfScope ps(ctx, BMND_KERNEL_REDUCE, st);
        launch_reduce(D, dj, nj, t.vox, 0, rgrid, st);
      }
      CU(cudaGetLastError());
    }
  }
  return BMND_OK;
}

// Scratch layout of several arrays: the synthesis caches of mass-conserving
// jobs when they fit `budget` (0: no limit), job i at offset base[i].
size_t layout_jobs(std::vector<Plan> &plans, const std::vector<JobIO> &io, size_t budget, std::vector<size_t> &base) {
  const int nj = (int)plans.size();
  for (int i = 0; i < nj; ++i)
    if (io[i].mass_conserve) add_mc_cache(plans[i]);
  base.assign(nj, 0);
  size_t need = 0;
  for (int pass = 0; pass < 2; ++pass) {
    need = 0;
    for (int i = 0; i < nj; ++i) { base[i] = need; need = al256(need + plans[i].total); }
    if (!budget || need <= budget) break;
    for (auto &pl : plans) drop_mc_cache(pl);
  }
  return need;
}

}  // namespace

// A recorded call (bmnd_graph_create): its own scratch, descriptor table and
// tile counter, and the instantiated graph of its launches.
struct bmnd_graph {
  int device = 0;
  void *scratch = nullptr;
  DJob *dtab = nullptr;
  int *counter = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void graph_release(bmnd_graph *G) {
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->scratch) cudaFree(G->scratch);
  if (G->dtab) cudaFree(G->dtab);
  if (G->counter) cudaFree(G->counter);
  delete G;
}

// Run both requested stages of several arrays with shared launches.  All
// plans must have the same kernel rank D.  first_stage/last_stage select a
// sub-range (bmnd_stage runs one stage with an external pilot).
bmnd_status run_jobs(bmnd_ctx *ctx, std::vector<Plan> &plans, const std::vector<JobIO> &io,
                     const bmnd_params &pr, int first_stage, int last_stage, const float *ext_pilot,
                     cudaStream_t st) {
  const int D = plans[0].D;
  bool mixed = false;
  for (auto &pl : plans) mixed = mixed || pl.D != D;
  if (mixed) {
    // jobs of different ranks run one rank class after another on the same
    // stream (the stage kernels are compiled per rank); each class is one
    // persistent launch per kernel as for a batch of one rank
    for (int d = 1; d <= KMAXD; ++d) {
      std::vector<Plan> sub;
      std::vector<JobIO> sio;
      for (size_t i = 0; i < plans.size(); ++i)
        if (plans[i].D == d) {
          sub.push_back(plans[i]);
          sio.push_back(io[i]);
        }
      if (sub.empty()) continue;
      bmnd_status rc = run_jobs(ctx, sub, sio, pr, first_stage, last_stage, nullptr, st);
      if (rc != BMND_OK) return rc;
    }
    return BMND_OK;
  }
  std::vector<size_t> base;
  const size_t need = layout_jobs(plans, io, ctx->budget, base);
  bmnd_status rc = ensure_arena(ctx, need, st);
  if (rc != BMND_OK) return rc;
  char *A = (char *)ctx->arena;
  JobTables t;
  build_tables(plans, io, pr, first_stage, last_stage, ext_pilot, A, base, t);
  rc = stage_jobs(ctx, t.h, st);
  if (rc != BMND_OK) return rc;
  return record_launches(ctx, plans, t, A, base, first_stage, last_stage, ctx->djobs, ctx->counters, st);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void bmnd_default_params(bmnd_params *p) {
  if (!p) return;
  p->lambda_ht = 3.0;
  p->gamma_ht = 3.0;
  p->gamma_wie = 0.0;
  p->tau_ht = 0.0;
  p->tau_wie = 0.0;
  p->s_v = 0.4;
  p->kaiser_beta = 2.0;
  p->shift_density = 2.0;
  p->passes = 2;
  p->schedule = BMND_SCHEDULE_GENERATED;
  p->power_mode = BMND_POWER_CLASSIC;
  p->group_transform = BMND_GROUP_HAAR;
  p->min_group = 2;
  p->weight_model = BMND_WEIGHT_VARIANCE;
  p->weight_scope = BMND_SCOPE_PATCH;
  p->match_metric = BMND_METRIC_SSD;
  p->match_policy = BMND_POLICY_FIXED;
  p->match_t = 3.0;
  p->beta_s = 0.1;
  p->kappa_s = 1.0;
  p->ht_rule = BMND_HT_HARD;
  p->weight_domain = BMND_DOMAIN_COEFFICIENT;
  p->cov_planes = 0;
  p->spatial_transform = BMND_SPATIAL_DCT;
}

bmnd_status bmnd_create(bmnd_ctx **out, int device, size_t scratch_budget_bytes) {
  if (!out) return BMND_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return BMND_EINVAL;
  }
  bmnd_ctx *ctx = new bmnd_ctx();
  ctx->device = device;
  ctx->budget = scratch_budget_bytes;
  bmnd_status rc = BMND_OK;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = BMND_ECUDA; break; }
    if (cudaDeviceGetAttribute(&ctx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      rc = BMND_ECUDA;
      break;
    }
    rc = init_constants(ctx);
    if (rc != BMND_OK) break;
    // the static tile counter of the persistent kernel shares the CTA's shared memory
    ctx->max_smem -= 64;
    if (cudaMalloc(&ctx->counters, 64 * sizeof(int)) != cudaSuccess) { rc = BMND_ENOMEM; break; }
    if (cudaMalloc(&ctx->diag, 4 * sizeof(unsigned long long)) != cudaSuccess) { rc = BMND_ENOMEM; break; }
    if (cudaMemset(ctx->diag, 0, 4 * sizeof(unsigned long long)) != cudaSuccess) { rc = BMND_ECUDA; break; }
    std::vector<unsigned char> t;
    fill_tables(t);
    if (cudaMalloc(&ctx->tab, t.size()) != cudaSuccess) { rc = BMND_ENOMEM; break; }
    ctx->tab64 = reinterpret_cast<const double *>(reinterpret_cast<unsigned char *>(ctx->tab) + TAB64_OFFSET);
    if (cudaMemcpy(ctx->tab, t.data(), t.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = BMND_ECUDA;
      break;
    }
    if (cudaEventCreateWithFlags(&ctx->staged, cudaEventDisableTiming) != cudaSuccess) { rc = BMND_ECUDA; break; }
  } while (0);
  if (rc != BMND_OK) {
    cudaGetLastError();
    bmnd_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return BMND_OK;
}

bmnd_status bmnd_set_profiling(bmnd_ctx *ctx, int enable) {
  if (!ctx) return BMND_EINVAL;
  ctx->profiling = enable != 0;
  return BMND_OK;
}

bmnd_status bmnd_kernel_stats(bmnd_ctx *ctx, int kind, int reset, int64_t *launches, double *total_ms) {
  if (!ctx) return BMND_EINVAL;
  if (kind < 0 || kind >= BMND_KERNEL_KINDS) return fail(ctx, BMND_EINVAL, "unknown kernel kind %d", kind);
  CU(cudaSetDevice(ctx->device));
  CU(cudaDeviceSynchronize());
  for (auto &m : ctx->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
      ctx->k_ms[m.kind] += ms;
      ctx->k_launches[m.kind] += 1;
    }
    ctx->event_pool.push_back(m.a);
    ctx->event_pool.push_back(m.b);
  }
  ctx->marks.clear();
  if (launches) *launches = ctx->k_launches[kind];
  if (total_ms) *total_ms = ctx->k_ms[kind];
  if (reset)
    for (int k = 0; k < BMND_KERNEL_KINDS; ++k) { ctx->k_launches[k] = 0; ctx->k_ms[k] = 0; }
  return BMND_OK;
}

bmnd_status bmnd_decision_stats(bmnd_ctx *ctx, int reset, uint64_t counts[3]) {
  if (!ctx || !counts) return BMND_EINVAL;
  CU(cudaSetDevice(ctx->device));
  CU(cudaDeviceSynchronize());
  unsigned long long h[4] = {0, 0, 0, 0};
  CU(cudaMemcpy(h, ctx->diag, sizeof(h), cudaMemcpyDeviceToHost));
  for (int k = 0; k < 3; ++k) counts[k] = h[k];
  if (reset) CU(cudaMemset(ctx->diag, 0, sizeof(h)));
  return BMND_OK;
}

bmnd_status bmnd_destroy(bmnd_ctx *ctx) {
  if (!ctx) return BMND_EINVAL;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto &m : ctx->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->tab) cudaFree(ctx->tab);
  if (ctx->diag) cudaFree(ctx->diag);
  if (ctx->hio) cudaFree(ctx->hio);
  if (ctx->counters) cudaFree(ctx->counters);
  if (ctx->djobs) cudaFree(ctx->djobs);
  if (ctx->hjobs) cudaFreeHost(ctx->hjobs);
  if (ctx->staged) cudaEventDestroy(ctx->staged);
  for (auto m : ctx->mom)
    if (m) cudaFree(m);
  for (auto m : ctx->pfix)
    if (m) cudaFree(m);
  delete ctx;
  return BMND_OK;
}

const char *bmnd_last_error(const bmnd_ctx *ctx) { return ctx ? ctx->err : "null context"; }

bmnd_status bmnd_match_moments(int metric, int count, float *mu, float *v) {
  if (metric < BMND_METRIC_DEVIANCE || metric > BMND_METRIC_ANSCOMBE || count < 1 || count > BMND_MOMENT_NMAX + 1 ||
      !mu || !v)
    return BMND_EINVAL;
  std::vector<float2> h;
  moment_table(metric, count, h);
  for (int n = 0; n < count; ++n) {
    mu[n] = h[n].x;
    v[n] = h[n].y;
  }
  return BMND_OK;
}

bmnd_status bmnd_denoise_ex(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape,
                            bmnd_noise noise, const int *patch, const int *step, const int *search,
                            const int *group_size, int stages, int mass_conserve,
                            const bmnd_params *params, float *out, void *stream) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (!y || !out) return fail(ctx, BMND_EINVAL, "null y or out");
  if (!group_size) return fail(ctx, BMND_EINVAL, "null group_size");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  bmnd_status rc = check_noise(ctx, noise, &pr);
  if (rc != BMND_OK) return rc;
  if (mass_conserve < 0 || mass_conserve > 3) return fail(ctx, BMND_EINVAL, "mass_conserve must be in [0, 3]");
  CU(cudaSetDevice(ctx->device));
  std::vector<Plan> plans(1);
  rc = make_plan(ctx, ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr, plans[0]);
  if (rc != BMND_OK) return rc;
  int64_t N = plans[0].g.N;
  if (!(y + N <= out || out + N <= y)) return fail(ctx, BMND_EINVAL, "out overlaps y");
  JobIO io{y, out, noise, {group_size[0], stages == 2 ? group_size[1] : group_size[0]}, stages,
           mass_conserve & (stages == 2 ? 3 : 1)};
  return run_jobs(ctx, plans, {io}, pr, 1, stages, nullptr, (cudaStream_t)stream);
}

bmnd_status bmnd_denoise(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape,
                         bmnd_noise noise, const int *patch, const int *step, const int *search,
                         const int *group_size, int stages, int mass_conserve, float *out,
                         void *stream) {
  return bmnd_denoise_ex(ctx, y, ndim, shape, noise, patch, step, search, group_size, stages,
                         mass_conserve, nullptr, out, stream);
}

// Tile cores the tuners time for a plan: the planner's core first, powers
// of two per axis for one or two axes, steps of one and two around the
// planner's core for more.
// Whether a plan's stage launches would run two CTAs per SM by shared memory
// (the tuners then also time one CTA per SM, with the full register file).
bool two_ctas_possible(const Plan &pl) {
  const int s = std::max(pl.smem[0], pl.smem[1]);
  return 2 * (s + 1024) <= 233472;
}

std::vector<std::vector<int>> tune_candidates(const Plan &p0) {
  const int D = p0.D;
  std::vector<std::vector<int>> cand;
  auto add = [&](std::vector<int> c) {
    for (int a = 0; a < D; ++a) c[a] = (int)std::max<int64_t>(1, std::min<int64_t>(c[a], p0.g.ell[a] + 1));
    if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
  };
  std::vector<int> def(D);
  for (int a = 0; a < D; ++a) def[a] = p0.g.C[a];
  add(def);
  if (D == 1) {
    for (int v : {16, 32, 64, 128, 256, 512}) add({v});
  } else if (D == 2) {
    for (int v0 : {4, 8, 16, 32})
      for (int v1 : {4, 8, 16, 32}) add({v0, v1});
  } else {
    for (int a = 0; a < D; ++a)
      for (int dl : {-2, -1, 1, 2}) {
        std::vector<int> c = def;
        c[a] += dl;
        if (c[a] >= 1) add(c);
      }
  }
  return cand;
}

bmnd_status bmnd_autotune(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape, bmnd_noise noise,
                          const int *patch, const int *step, const int *search, const int *group_size, int stages,
                          int mass_conserve, const bmnd_params *params, float *out, void *stream, int *core) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (!y || !out) return fail(ctx, BMND_EINVAL, "null y or out");
  if (!group_size) return fail(ctx, BMND_EINVAL, "null group_size");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  bmnd_status rc = check_noise(ctx, noise, &pr);
  if (rc != BMND_OK) return rc;
  if (mass_conserve < 0 || mass_conserve > 3) return fail(ctx, BMND_EINVAL, "mass_conserve must be in [0, 3]");
  CU(cudaSetDevice(ctx->device));
  const std::string key = tune_key(ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr);
  ctx->tuned.erase(key);
  std::vector<Plan> plans(1);
  rc = make_plan(ctx, ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr, plans[0]);
  if (rc != BMND_OK) return rc;
  const Plan &p0 = plans[0];
  const int D = p0.D;
  const int64_t N = p0.g.N;
  if (!(y + N <= out || out + N <= y)) return fail(ctx, BMND_EINVAL, "out overlaps y");
  std::vector<std::vector<int>> cand = tune_candidates(p0);
  std::vector<int> def = cand[0];
  const JobIO io{y, out, noise, {group_size[0], stages == 2 ? group_size[1] : group_size[0]}, stages,
                 mass_conserve & (stages == 2 ? 3 : 1)};
  const std::vector<JobIO> ios{io};
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  double best_ms = 1e30;
  std::vector<int> best = def;
  // every core also with one CTA per SM (the full register file) where the
  // shared memory would allow two
  const size_t ncore = cand.size();
  for (size_t i = 0; i < ncore; ++i) {
    std::vector<int> c1 = cand[i];
    c1.push_back(1);
    cand.push_back(c1);
  }
  for (const std::vector<int> &c : cand) {
    ctx->force_core = &c;
    std::vector<Plan> pc(1);
    rc = make_plan(ctx, ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr, pc[0]);
    if (rc != BMND_OK) break;
    bool fits = true;
    for (int a = 0; a < D; ++a) fits = fits && pc[0].g.C[a] == c[a];
    if (!fits || ((int)c.size() > D && !two_ctas_possible(pc[0]))) continue;
    // one untimed run, then two timed ones
    rc = run_jobs(ctx, pc, ios, pr, 1, stages, nullptr, st);
    if (rc != BMND_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && rc == BMND_OK; ++r) rc = run_jobs(ctx, pc, ios, pr, 1, stages, nullptr, st);
    if (rc != BMND_OK) break;
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = fail(ctx, BMND_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  ctx->force_core = nullptr;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != BMND_OK) return rc;
  ctx->tuned[key] = best;
  // the tuned estimate in out
  std::vector<Plan> pf(1);
  rc = make_plan(ctx, ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr, pf[0]);
  if (rc == BMND_OK) rc = run_jobs(ctx, pf, ios, pr, 1, stages, nullptr, st);
  if (rc == BMND_OK && core) {
    for (int d = 0; d < ndim; ++d) core[d] = 1;
    for (int a = 0; a < D; ++a) core[pf[0].kax_of[a]] = pf[0].g.C[a];
  }
  return rc;
}

bmnd_status bmnd_graph_create(bmnd_ctx *ctx, const float *y, int ndim, const int64_t *shape, bmnd_noise noise,
                              const int *patch, const int *step, const int *search, const int *group_size,
                              int stages, int mass_conserve, const bmnd_params *params, float *out,
                              bmnd_graph **graph) {
  if (!ctx || !graph) return BMND_EINVAL;
  *graph = nullptr;
  ctx->err[0] = 0;
  if (!y || !out) return fail(ctx, BMND_EINVAL, "null y or out");
  if (!group_size) return fail(ctx, BMND_EINVAL, "null group_size");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  bmnd_status rc = check_noise(ctx, noise, &pr);
  if (rc != BMND_OK) return rc;
  if (mass_conserve < 0 || mass_conserve > 3) return fail(ctx, BMND_EINVAL, "mass_conserve must be in [0, 3]");
  CU(cudaSetDevice(ctx->device));
  std::vector<Plan> plans(1);
  rc = make_plan(ctx, ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr, plans[0]);
  if (rc != BMND_OK) return rc;
  const int64_t N = plans[0].g.N;
  if (!(y + N <= out || out + N <= y)) return fail(ctx, BMND_EINVAL, "out overlaps y");
  JobIO io{y, out, noise, {group_size[0], stages == 2 ? group_size[1] : group_size[0]}, stages,
           mass_conserve & (stages == 2 ? 3 : 1)};
  std::vector<JobIO> ios{io};
  std::vector<size_t> base;
  const size_t need = layout_jobs(plans, ios, ctx->budget, base);
  bmnd_graph *G = new bmnd_graph();
  G->device = ctx->device;
  if (cudaMalloc(&G->scratch, std::max<size_t>(need, 256)) != cudaSuccess ||
      cudaMalloc(&G->dtab, 2 * sizeof(DJob)) != cudaSuccess || cudaMalloc(&G->counter, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    graph_release(G);
    return fail(ctx, BMND_ENOMEM, "graph scratch of %zu bytes could not be allocated", need);
  }
  JobTables t;
  build_tables(plans, ios, pr, 1, stages, nullptr, (char *)G->scratch, base, t);
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaMemcpy(G->dtab, t.h.data(), 2 * sizeof(DJob), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (cs) cudaStreamDestroy(cs);
    graph_release(G);
    return fail(ctx, BMND_ECUDA, "graph set-up: %s", cudaGetErrorString(e));
  }
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  rc = record_launches(ctx, plans, t, (char *)G->scratch, base, 1, stages, G->dtab, G->counter, cs);
  ctx->profiling = prof;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  if (rc == BMND_OK && e == cudaSuccess) e = cudaGraphInstantiate(&G->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (rc != BMND_OK || e != cudaSuccess) {
    cudaGetLastError();
    graph_release(G);
    if (rc != BMND_OK) return rc;
    return fail(ctx, BMND_ECUDA, "graph recording: %s", cudaGetErrorString(e));
  }
  *graph = G;
  return BMND_OK;
}

bmnd_status bmnd_graph_launch(bmnd_graph *graph, void *stream) {
  if (!graph || !graph->exec) return BMND_EINVAL;
  if (cudaSetDevice(graph->device) != cudaSuccess ||
      cudaGraphLaunch(graph->exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return BMND_ECUDA;
  }
  return BMND_OK;
}

bmnd_status bmnd_graph_destroy(bmnd_graph *graph) {
  if (!graph) return BMND_EINVAL;
  cudaSetDevice(graph->device);
  cudaDeviceSynchronize();
  graph_release(graph);
  return BMND_OK;
}

bmnd_status bmnd_stage(bmnd_ctx *ctx, const float *y, const float *pilot, int ndim,
                       const int64_t *shape, bmnd_noise noise, const int *patch, const int *step,
                       const int *search, int group_max, int stage, int mass_conserve,
                       const bmnd_params *params, float *out, void *stream) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (!y || !out) return fail(ctx, BMND_EINVAL, "null y or out");
  if (stage != 1 && stage != 2) return fail(ctx, BMND_EINVAL, "stage must be 1 or 2");
  if (stage == 2 && !pilot) return fail(ctx, BMND_EINVAL, "stage 2 needs a pilot");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  bmnd_status rc = check_noise(ctx, noise, &pr);
  if (rc != BMND_OK) return rc;
  CU(cudaSetDevice(ctx->device));
  int gs[2] = {group_max, group_max};
  std::vector<Plan> plans(1);
  int mc = mass_conserve ? (stage == 1 ? 1 : 2) : 0;
  rc = make_plan(ctx, ndim, shape, patch, step, search, gs, stage, mc, pr, plans[0]);
  if (rc != BMND_OK) return rc;
  int64_t N = plans[0].g.N;
  if (!(y + N <= out || out + N <= y)) return fail(ctx, BMND_EINVAL, "out overlaps y");
  if (pilot && !(pilot + N <= out || out + N <= pilot)) return fail(ctx, BMND_EINVAL, "out overlaps pilot");
  JobIO io{y, out, noise, {group_max, group_max}, stage, mc};
  return run_jobs(ctx, plans, {io}, pr, stage, stage, pilot, (cudaStream_t)stream);
}

static bmnd_status match_or_schedule(bmnd_ctx *ctx, const float *guide, int ndim, const int64_t *shape,
                                      bmnd_noise noise, const int *patch, const int *step,
                                      const int *search, int group_max, int stage,
                                      const bmnd_params *params, int64_t *origins, int64_t *groups,
                                      int32_t *counts, int64_t cap, int64_t *n_refs, void *stream,
                                      bool do_match) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (!n_refs || !origins) return fail(ctx, BMND_EINVAL, "null origins or n_refs");
  if (do_match && (!guide || !groups || !counts)) return fail(ctx, BMND_EINVAL, "null guide/groups/counts");
  if (do_match && stage != 1 && stage != 2) return fail(ctx, BMND_EINVAL, "stage must be 1 or 2");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  if (do_match) {
    bmnd_status rc = check_noise(ctx, noise, &pr);
    if (rc != BMND_OK) return rc;
  }
  static const int ones[BMND_MAX_NDIM] = {1, 1, 1, 1, 1, 1, 1, 1};
  if (!do_match) search = ones;
  cudaStream_t st = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  int gs[2] = {do_match ? group_max : 1, do_match ? group_max : 1};
  Plan pl;
  bmnd_status rc = make_plan(ctx, ndim, shape, patch, step, search, gs, do_match && stage == 2 ? 2 : 1, 0,
                             pr, pl);
  if (rc != BMND_OK) return rc;
  size_t tileoff_bytes = al256((size_t)pl.g.ntiles * 8);
  rc = ensure_arena(ctx, pl.total + tileoff_bytes, st);
  if (rc != BMND_OK) return rc;
  char *B = (char *)ctx->arena;
  DJob J;
  memset(&J, 0, sizeof(J));
  J.g = pl.g;
  fill_stage(J.g, stage == 2 ? 2 : 1, gs[0], noise, pr);
  J.y = guide;
  J.guide = guide;
  J.ref_local = (const int *)(B + pl.o_refs);
  J.ref_count = (const int *)(B + pl.o_rcount);
  J.groups = (int *)(B + pl.o_groups);
  J.gcount = (int *)(B + pl.o_gcount);
  std::vector<DJob> h{J};
  rc = stage_jobs(ctx, h, st);
  if (rc != BMND_OK) return rc;
  CU(cudaMemsetAsync(B + pl.o_flags, 0, (size_t)pl.nflags, st));
  launch_sched(pl.s, (unsigned char *)(B + pl.o_flags), ctx->djobs, pl.g.ntiles, (int *)(B + pl.o_refs),
               (int *)(B + pl.o_rcount), st);
  CU(cudaGetLastError());
  if (do_match) {
    int sm = stage_smem(J.g, gs[0], J.g.stage == 2 ? 2 : 1, false, J.g.stage != 2);
    ProfScope ps(ctx, BMND_KERNEL_MATCH, st);
    rc = launch_stage(ctx, pl.D, kernel_jl(pl), pick_kb(pl), stage == 2 ? 2 : kernel_stage(pl.metric, 1), ctx->djobs,
                      1, pl.g.ntiles, 1, sm, st);
    if (rc != BMND_OK) return rc;
  }
  std::vector<int> cnt(pl.g.ntiles);
  CU(cudaMemcpyAsync(cnt.data(), B + pl.o_rcount, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  std::vector<int64_t> off(pl.g.ntiles);
  int64_t tot = 0;
  for (int t = 0; t < pl.g.ntiles; ++t) { off[t] = tot; tot += cnt[t]; }
  *n_refs = tot;
  int64_t *doff = (int64_t *)(B + pl.total);
  CU(cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, st));
  launch_export(pl.D, ctx->djobs, pl.g.ntiles, doff, origins, do_match ? groups : nullptr,
                do_match ? counts : nullptr, cap, st);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  if (tot > cap) return fail(ctx, BMND_ENOMEM, "capacity %lld < %lld references", (long long)cap, (long long)tot);
  return BMND_OK;
}

bmnd_status bmnd_schedule(bmnd_ctx *ctx, int ndim, const int64_t *shape, const int *patch,
                          const int *step, const bmnd_params *params, int64_t *origins,
                          int64_t cap, int64_t *n_refs, void *stream) {
  bmnd_noise nz{BMND_NOISE_GAUSSIAN, 0.0, 1.0};
  return match_or_schedule(ctx, nullptr, ndim, shape, nz, patch, step, nullptr, 1, 1, params, origins,
                           nullptr, nullptr, cap, n_refs, stream, false);
}

bmnd_status bmnd_coverage(bmnd_ctx *ctx, int ndim, const int64_t *shape, const int *patch, const int *step,
                          const bmnd_params *params, int32_t *coverage, int64_t *n_refs, double *cv, void *stream) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (!n_refs || !cv) return fail(ctx, BMND_EINVAL, "null n_refs or cv");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  static const int ones[BMND_MAX_NDIM] = {1, 1, 1, 1, 1, 1, 1, 1};
  cudaStream_t st = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  int gs[2] = {1, 1};
  Plan pl;
  bmnd_status rc = make_plan(ctx, ndim, shape, patch, step, ones, gs, 1, 0, pr, pl);
  if (rc != BMND_OK) return rc;
  const size_t o_sums = al256(pl.o_flags + (size_t)pl.nflags);
  rc = ensure_arena(ctx, o_sums + 3 * sizeof(unsigned long long), st);
  if (rc != BMND_OK) return rc;
  unsigned char *B = (unsigned char *)ctx->arena;
  unsigned long long *sums = (unsigned long long *)(B + o_sums);
  CovGeom c;
  memset(&c, 0, sizeof(c));
  c.D = pl.D;
  c.P = pl.g.P;
  c.N = pl.g.N;
  c.nflags = pl.nflags;
  for (int a = 0; a < pl.D; ++a) {
    c.L[a] = pl.g.L[a];
    c.ell[a] = pl.g.ell[a];
    c.fst[a] = pl.s.fst[a];
    c.j[a] = pl.g.j[a];
  }
  {
    ProfScope ps(ctx, BMND_KERNEL_SCHEDULE, st);
    CU(cudaMemsetAsync(B + pl.o_flags, 0, (size_t)pl.nflags, st));
    CU(cudaMemsetAsync(sums, 0, 3 * sizeof(unsigned long long), st));
    launch_sched_mark(pl.s, B + pl.o_flags, st);
    launch_coverage(c, B + pl.o_flags, coverage, sums, st);
    CU(cudaGetLastError());
  }
  unsigned long long h[3];
  CU(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *n_refs = (int64_t)h[2];
  const double mu = (double)h[0] / (double)c.N;
  const double var = (double)h[1] / (double)c.N - mu * mu;
  *cv = mu > 0 ? std::sqrt(std::max(var, 0.0)) / mu : 0.0;
  return BMND_OK;
}

bmnd_status bmnd_match(bmnd_ctx *ctx, const float *guide, int ndim, const int64_t *shape,
                       bmnd_noise noise, const int *patch, const int *step, const int *search,
                       int group_max, int stage, const bmnd_params *params, int64_t *origins,
                       int64_t *groups, int32_t *counts, int64_t cap, int64_t *n_refs,
                       void *stream) {
  return match_or_schedule(ctx, guide, ndim, shape, noise, patch, step, search, group_max, stage, params,
                           origins, groups, counts, cap, n_refs, stream, true);
}

bmnd_status bmnd_denoise_batch(bmnd_ctx *ctx, int n_jobs, const bmnd_job *jobs,
                               const bmnd_params *params, void *stream) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (n_jobs < 1 || !jobs) return fail(ctx, BMND_EINVAL, "no jobs");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  CU(cudaSetDevice(ctx->device));
  std::vector<Plan> plans(n_jobs);
  std::vector<JobIO> io(n_jobs);
  int stages = jobs[0].stages;
  for (int i = 0; i < n_jobs; ++i) {
    const bmnd_job &jb = jobs[i];
    if (!jb.y || !jb.out) return fail(ctx, BMND_EINVAL, "job %d: null y or out", i);
    bmnd_status rc = check_noise(ctx, jb.noise, &pr);
    if (rc != BMND_OK) return rc;
    if (jb.stages != stages) return fail(ctx, BMND_EUNSUPPORTED, "job %d: all jobs must use the same stage count", i);
    if (jb.mass_conserve < 0 || jb.mass_conserve > 3) return fail(ctx, BMND_EINVAL, "job %d: bad mass_conserve", i);
    rc = make_plan(ctx, jb.ndim, jb.shape, jb.patch, jb.step, jb.search, jb.group_size, jb.stages,
                   jb.mass_conserve, pr, plans[i]);
    if (rc != BMND_OK) return rc;
    int64_t N = plans[i].g.N;
    if (!(jb.y + N <= jb.out || jb.out + N <= jb.y)) return fail(ctx, BMND_EINVAL, "job %d: out overlaps y", i);
    io[i] = JobIO{jb.y, jb.out, jb.noise, {jb.group_size[0], stages == 2 ? jb.group_size[1] : jb.group_size[0]},
                  stages, jb.mass_conserve & (stages == 2 ? 3 : 1)};
  }
  return run_jobs(ctx, plans, io, pr, 1, stages, nullptr, (cudaStream_t)stream);
}

bmnd_status bmnd_autotune_batch(bmnd_ctx *ctx, int n_jobs, const bmnd_job *jobs, const bmnd_params *params,
                                void *stream, int *core) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (n_jobs < 1 || !jobs) return fail(ctx, BMND_EINVAL, "no jobs");
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  CU(cudaSetDevice(ctx->device));
  const int stages = jobs[0].stages;
  std::vector<JobIO> io(n_jobs);
  std::vector<std::string> keys(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    const bmnd_job &jb = jobs[i];
    if (!jb.y || !jb.out) return fail(ctx, BMND_EINVAL, "job %d: null y or out", i);
    bmnd_status rc = check_noise(ctx, jb.noise, &pr);
    if (rc != BMND_OK) return rc;
    if (jb.stages != stages) return fail(ctx, BMND_EUNSUPPORTED, "job %d: all jobs must use the same stage count", i);
    if (jb.mass_conserve < 0 || jb.mass_conserve > 3) return fail(ctx, BMND_EINVAL, "job %d: bad mass_conserve", i);
    keys[i] = tune_key(jb.ndim, jb.shape, jb.patch, jb.step, jb.search, jb.group_size, jb.stages, jb.mass_conserve, pr);
    io[i] = JobIO{jb.y, jb.out, jb.noise, {jb.group_size[0], stages == 2 ? jb.group_size[1] : jb.group_size[0]},
                  stages, jb.mass_conserve & (stages == 2 ? 3 : 1)};
  }
  // the jobs sharing the first job's problem key are tuned together
  const std::string key = keys[0];
  ctx->tuned.erase(key);
  auto plan_all = [&](const std::vector<int> *c, std::vector<Plan> &plans) -> bmnd_status {
    plans.assign(n_jobs, Plan());
    for (int i = 0; i < n_jobs; ++i) {
      const bmnd_job &jb = jobs[i];
      ctx->force_core = keys[i] == key ? c : nullptr;
      bmnd_status rc = make_plan(ctx, jb.ndim, jb.shape, jb.patch, jb.step, jb.search, jb.group_size, jb.stages,
                                 jb.mass_conserve, pr, plans[i]);
      ctx->force_core = nullptr;
      if (rc != BMND_OK) return rc;
      const int64_t N = plans[i].g.N;
      if (!(jb.y + N <= jb.out || jb.out + N <= jb.y)) return fail(ctx, BMND_EINVAL, "job %d: out overlaps y", i);
    }
    return BMND_OK;
  };
  std::vector<Plan> plans;
  bmnd_status rc = plan_all(nullptr, plans);
  if (rc != BMND_OK) return rc;
  const std::vector<std::vector<int>> cand = tune_candidates(plans[0]);
  const int D = plans[0].D;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  double best_ms = 1e30;
  std::vector<int> best = cand[0];
  std::vector<std::vector<int>> cands = cand;
  for (const std::vector<int> &c0 : cand) {
    std::vector<int> c1 = c0;
    c1.push_back(1);
    cands.push_back(c1);
  }
  for (const std::vector<int> &c : cands) {
    rc = plan_all(&c, plans);
    if (rc != BMND_OK) break;
    bool fits = true;
    for (int a = 0; a < D; ++a) fits = fits && plans[0].g.C[a] == c[a];
    if (!fits || ((int)c.size() > D && !two_ctas_possible(plans[0]))) continue;
    // one untimed batch, then two timed ones
    rc = run_jobs(ctx, plans, io, pr, 1, stages, nullptr, st);
    if (rc != BMND_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && rc == BMND_OK; ++r) rc = run_jobs(ctx, plans, io, pr, 1, stages, nullptr, st);
    if (rc != BMND_OK) break;
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rc = fail(ctx, BMND_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != BMND_OK) return rc;
  ctx->tuned[key] = best;
  rc = plan_all(nullptr, plans);
  if (rc == BMND_OK) rc = run_jobs(ctx, plans, io, pr, 1, stages, nullptr, st);
  if (rc == BMND_OK && core) {
    for (int d = 0; d < jobs[0].ndim; ++d) core[d] = 1;
    for (int a = 0; a < D; ++a) core[plans[0].kax_of[a]] = plans[0].g.C[a];
  }
  return rc;
}

bmnd_status bmnd_denoise_batch_host(bmnd_ctx *ctx, int n_jobs, const bmnd_job *jobs, const bmnd_params *params,
                                    void *stream) {
  if (!ctx) return BMND_EINVAL;
  ctx->err[0] = 0;
  if (n_jobs < 1 || !jobs) return fail(ctx, BMND_EINVAL, "no jobs");
  CU(cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> n(n_jobs);
  size_t total = 0;
  for (int i = 0; i < n_jobs; ++i) {
    const bmnd_job &jb = jobs[i];
    if (!jb.y || !jb.out) return fail(ctx, BMND_EINVAL, "job %d: null y or out", i);
    if (jb.ndim < 1 || jb.ndim > BMND_MAX_NDIM) return fail(ctx, BMND_EINVAL, "job %d: bad ndim", i);
    int64_t c = 1;
    for (int d = 0; d < jb.ndim; ++d) {
      if (jb.shape[d] < 1) return fail(ctx, BMND_EINVAL, "job %d: bad shape", i);
      c *= jb.shape[d];
    }
    n[i] = c;
    total += 2 * (size_t)((c + 63) & ~(int64_t)63);
  }
  if (total > ctx->hio_floats) {
    CU(cudaStreamSynchronize(st));
    if (ctx->hio) CU(cudaFree(ctx->hio));
    ctx->hio = nullptr;
    ctx->hio_floats = 0;
    if (cudaMalloc(&ctx->hio, total * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, BMND_ENOMEM, "cudaMalloc of %zu bytes for the host path failed", total * sizeof(float));
    }
    ctx->hio_floats = total;
  }
  std::vector<bmnd_job> dj(jobs, jobs + n_jobs);
  size_t off = 0;
  for (int i = 0; i < n_jobs; ++i) {
    float *dy = ctx->hio + off, *dout = dy + ((n[i] + 63) & ~(int64_t)63);
    off += 2 * (size_t)((n[i] + 63) & ~(int64_t)63);
    CU(cudaMemcpyAsync(dy, jobs[i].y, n[i] * sizeof(float), cudaMemcpyHostToDevice, st));
    dj[i].y = dy;
    dj[i].out = dout;
  }
  bmnd_status rc = bmnd_denoise_batch(ctx, n_jobs, dj.data(), params, stream);
  if (rc != BMND_OK) return rc;
  for (int i = 0; i < n_jobs; ++i)
    CU(cudaMemcpyAsync(jobs[i].out, dj[i].out, n[i] * sizeof(float), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  return BMND_OK;
}

bmnd_status bmnd_plan_info(bmnd_ctx *ctx, int ndim, const int64_t *shape, const int *patch, const int *step,
                           const int *search, const int *group_size, int stages, int mass_conserve,
                           const bmnd_params *params, int64_t info[8]) {
  if (!ctx || !info || !group_size) return BMND_EINVAL;
  ctx->err[0] = 0;
  bmnd_params pr;
  if (params) pr = *params; else bmnd_default_params(&pr);
  Plan pl;
  bmnd_status rc = make_plan(ctx, ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr, pl);
  if (rc != BMND_OK) return rc;
  info[0] = pl.g.ntiles;
  info[1] = pl.g.region;
  info[2] = pl.g.cap;
  info[3] = pl.D;
  for (int a = 0; a < 4; ++a) info[4 + a] = a < pl.D ? pl.g.C[a] : 0;
  return BMND_OK;
}

bmnd_status bmnd_fp32_fma_peak(int device, double *tflops) {
  if (!tflops) return BMND_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return BMND_EINVAL;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return BMND_ECUDA;
  float *out = nullptr;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) {
    cudaGetLastError();
    return BMND_ENOMEM;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a);
    launch_fma_peak(out, blocks, threads, iters);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && rep > 0) {
      const double flop = 2.0 * (double)FMA_PEAK_CHAINS * iters * blocks * threads;
      best = std::max(best, (float)(flop / (ms * 1e-3) / 1e12));
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BMND_ECUDA;
  }
  *tflops = best;
  return BMND_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free denoising
//
// For callers that must not allocate device memory: code that runs while
// another component owns the device allocator, inside a memory budget that is
// already spoken for, or in an environment where cudaMalloc is unavailable or
// would synchronize the device at the wrong moment.  The scratch of this entry
// point is one file-scope device array of fixed size, held by every GPU that
// loads the library until the process exits.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoallocBytes = (size_t)64 << 20;  // 64 MiB of scratch per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Layout of the array: [tile counter | job table (2 DJob) | DCT table | work].
constexpr size_t kNoallocCounter = 0;
constexpr size_t kNoallocJobs = 256;
constexpr size_t kNoallocTab = (kNoallocJobs + 2 * sizeof(DJob) + 255) & ~(size_t)255;
constexpr size_t kNoallocWork = (kNoallocTab + TAB_BYTES + 255) & ~(size_t)255;

struct NoallocDevice {
  bool ready;
  unsigned char *base;  // device address of g_noalloc_scratch on this device
  int max_smem;
  int num_sms;
};
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc[64];

// One-time set-up on the current device: resolve the array's device address,
// copy the transform tables (float and double DCT matrices) into it, upload
// the butterfly-DCT constants to the device's constant bank (the same ones
// bmnd_create uploads), read the SM count and shared-memory limit.
// Synchronous; the first call on a device must precede any stream capture.
bmnd_status noalloc_setup(int device, NoallocDevice *&out, char *err, size_t errlen) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (device < 0 || device >= 64) {
    snprintf(err, errlen, "device %d out of range", device);
    return BMND_EINVAL;
  }
  NoallocDevice &d = g_noalloc[device];
  if (!d.ready) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      snprintf(err, errlen, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      cudaGetLastError();
      return BMND_ECUDA;
    }
    std::vector<unsigned char> img;
    fill_tables(img);
    e = cudaMemcpy((unsigned char *)ptr + kNoallocTab, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = init_constants_on(device);
    int max_smem = 0, num_sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
      snprintf(err, errlen, "set-up: %s", cudaGetErrorString(e));
      cudaGetLastError();
      return BMND_ECUDA;
    }
    d.base = (unsigned char *)ptr;
    d.max_smem = max_smem - 64;
    d.num_sms = num_sms;
    d.ready = true;
  }
  out = &d;
  return BMND_OK;
}

// The allocation-free path on a stack context `c` whose scratch pointers lie
// in the static array (nothing in it allocates).
bmnd_status noalloc_run(bmnd_ctx *ctx, NoallocDevice *dev, const float *y, int ndim, const int64_t *shape,
                        bmnd_noise noise, const int *patch, const int *step, const int *search,
                        const int *group_size, int stages, int mass_conserve, float *out, cudaStream_t st) {
  if (!y || !out || !group_size) return fail(ctx, BMND_EINVAL, "null y, out or group_size");
  bmnd_status rc = check_noise(ctx, noise);
  if (rc != BMND_OK) return rc;
  if (mass_conserve < 0 || mass_conserve > 3) return fail(ctx, BMND_EINVAL, "mass_conserve must be in [0, 3]");
  bmnd_params pr;
  bmnd_default_params(&pr);
  Plan pl;
  rc = make_plan(ctx, ndim, shape, patch, step, search, group_size, stages, mass_conserve, pr, pl);
  if (rc != BMND_OK) return rc;
  const int64_t N = pl.g.N;
  if (!(y + N <= out || out + N <= y)) return fail(ctx, BMND_EINVAL, "out overlaps y");
  // the group tables (last in the plan's layout) are only used by mass
  // conservation
  const size_t need = kNoallocWork + (mass_conserve ? pl.total : pl.o_groups);
  if (need > kNoallocBytes)
    return fail(ctx, BMND_ENOMEM, "this array needs %zu bytes of scratch; the allocation-free entry point has %zu",
                need, kNoallocBytes);
  unsigned char *B = dev->base + kNoallocWork;
  const int gs1 = stages == 2 ? group_size[1] : group_size[0];
  const int mc = mass_conserve & (stages == 2 ? 3 : 1);
  DJob h[2];
  bool any_mc[2] = {false, false};
  int smax[2] = {0, 0};
  for (int s = 1; s <= 2; ++s) {
    DJob &J = h[s - 1];
    memset(&J, 0, sizeof(J));
    J.g = pl.g;
    fill_stage(J.g, s, s == 1 ? group_size[0] : gs1, noise, pr);
    const bool m = (mc >> (s - 1)) & 1;
    float *pilot = (float *)(B + pl.o_pilot);
    J.y = y;
    J.guide = s == 1 ? y : pilot;
    J.out = s == stages ? out : pilot;
    J.eta = m ? (float *)(B + pl.o_eta) : nullptr;
    J.partial = (float2 *)(B + pl.o_partial);
    J.ref_local = (const int *)(B + pl.o_refs);
    J.ref_count = (const int *)(B + pl.o_rcount);
    J.groups = m ? (int *)(B + pl.o_groups) : nullptr;
    J.gcount = m ? (int *)(B + pl.o_gcount) : nullptr;
    any_mc[s - 1] = m;
    smax[s - 1] = m ? std::max(pl.smem[s - 1], pl.smem[2]) : pl.smem[s - 1];
  }
  // from pageable host memory: the copy is staged before the call returns
  CU(cudaMemcpyAsync(ctx->djobs, h, sizeof(h), cudaMemcpyHostToDevice, st));
  // the schedule flags must start at zero; everything else the kernels read
  // (reference lists, partials, pilot, eta, group tables) is written first
  CU(cudaMemsetAsync(B + pl.o_flags, 0, (size_t)pl.nflags, st));
  launch_sched(pl.s, B + pl.o_flags, ctx->djobs, pl.g.ntiles, (int *)(B + pl.o_refs), (int *)(B + pl.o_rcount), st);
  CU(cudaGetLastError());
  const int64_t vox = pl.g.N;
  const int rgrid = (int)std::min<int64_t>((vox + 255) / 256, 148 * 32);
  for (int s = 1; s <= stages; ++s) {
    const DJob *dj = ctx->djobs + (s - 1);
    rc = launch_stage(ctx, pl.D, kernel_jl(pl), pick_kb(pl), s, dj, 1, pl.g.ntiles, 0, smax[s - 1], st,
                        nullptr, false, pl.minb);
    if (rc != BMND_OK) return rc;
    launch_reduce(pl.D, dj, 1, vox, any_mc[s - 1] ? 1 : 0, rgrid, st);
    CU(cudaGetLastError());
    if (any_mc[s - 1]) {
      rc = launch_stage(ctx, pl.D, kernel_jl(pl), pick_kb(pl), s, dj, 1, pl.g.ntiles, 2, smax[s - 1], st,
                        nullptr, false, pl.minb);
      if (rc != BMND_OK) return rc;
      launch_reduce(pl.D, dj, 1, vox, 0, rgrid, st);
      CU(cudaGetLastError());
    }
  }
  return BMND_OK;
}

}  // namespace

extern "C" {

bmnd_status bmnd_denoise_noalloc(const float *y, int ndim, const int64_t *shape, bmnd_noise noise,
                                 const int *patch, const int *step, const int *search,
                                 const int *group_size, int stages, int mass_conserve, float *out,
                                 void *stream, char *errbuf, size_t errlen) {
  char err[256] = {0};
  bmnd_status rc = BMND_OK;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    snprintf(err, sizeof(err), "no current CUDA device");
    rc = BMND_ECUDA;
  }
  if (rc == BMND_OK) {
    // the job table is copied from this call's stack: a recorded copy would
    // outlive it, so capture is refused
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cs) != cudaSuccess) {
      cudaGetLastError();
      snprintf(err, sizeof(err), "cudaStreamIsCapturing failed");
      rc = BMND_ECUDA;
    } else if (cs != cudaStreamCaptureStatusNone) {
      snprintf(err, sizeof(err), "the allocation-free entry point cannot be recorded by stream capture");
      rc = BMND_EUNSUPPORTED;
    }
  }
  NoallocDevice *dev = nullptr;
  if (rc == BMND_OK) rc = noalloc_setup(device, dev, err, sizeof(err));
  if (rc == BMND_OK) {
    bmnd_ctx c;  // pointers into the static array; nothing is allocated or freed
    c.device = device;
    c.max_smem = dev->max_smem;
    c.num_sms = dev->num_sms;
    c.counters = (int *)(dev->base + kNoallocCounter);
    c.djobs = (DJob *)(dev->base + kNoallocJobs);
    c.tab = (float *)(dev->base + kNoallocTab);
    c.tab64 = (const double *)(dev->base + kNoallocTab + TAB64_OFFSET);
    rc = noalloc_run(&c, dev, y, ndim, shape, noise, patch, step, search, group_size, stages, mass_conserve, out,
                     (cudaStream_t)stream);
    if (rc != BMND_OK) snprintf(err, sizeof(err), "%s", c.err);
  }
  if (errbuf && errlen) snprintf(errbuf, errlen, "%s", rc == BMND_OK ? "" : err);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving loop: memory-budgeted admission and continuous batching
// ---------------------------------------------------------------------------

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over the server's device arena (host bookkeeping).
struct ArenaAlloc {
  std::map<size_t, size_t> free_;  // offset -> size
  void init(size_t size) {
    free_.clear();
    free_[0] = size;
  }
  bool alloc(size_t bytes, size_t &off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        off = it->first;
        size_t rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

enum { SJ_PENDING = 0, SJ_STAGE1 = 1, SJ_STAGE2 = 2, SJ_DONE = 3, SJ_FAILED = 4 };

struct SrvJob {
  int64_t ticket = 0;
  bmnd_job spec;  // y / out are HOST pointers
  Plan plan;
  size_t off = 0, bytes = 0;
  int state = SJ_PENDING;
  bmnd_status status = BMND_OK;
  Clock::time_point t_submit, t_done;
  float *dy = nullptr, *dout = nullptr;
  DJob *djob = nullptr;        // this job's own descriptor (schedule kernels)
  unsigned char *scratch = nullptr;
  int lane = 0;                // 0 small jobs, 1 large jobs
  double est_ms = 0;           // estimated GPU time of both stages
  bool in_step = false;        // part of a step in flight
};

struct SrvStepRef {
  bmnd_server *S;
  int lane, slot;
};

// A step in flight: its jobs, the descriptor-table region it owns
// (2 x max_slots) and the flag its host callback sets at the end.
struct SrvStep {
  std::vector<SrvJob *> jobs;
  int tab_base = 0;
  bool busy = false, done = false;
  bmnd_status rc = BMND_OK;
  SrvStepRef ref;
};

// One lane of the server: its own stream (the small-job lane has the higher
// priority) and tile counter; up to two steps in flight, so that the next
// step is queued on the GPU while the host finishes the previous one.
struct SrvLane {
  cudaStream_t st = nullptr;
  int *counter = nullptr;
  bool tile_ctas = false;          // one CTA per tile (the large-job lane)
  std::vector<SrvJob *> active;    // admitted jobs, in a step or waiting for one
  SrvStep steps[2];
};

}  // namespace

struct bmnd_server {
  bmnd_ctx *ctx = nullptr;
  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  unsigned char *arena = nullptr;
  ArenaAlloc alloc;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<SrvJob *> pending;
  std::unordered_map<int64_t, SrvJob *> jobs;
  int64_t next_ticket = 1;
  std::thread worker;
  bool stop = false;
  bool admit_blocked = false;  // the oldest pending job waits for memory or a slot
  SrvLane lanes[2];
  cudaStream_t cst = nullptr;      // host <-> device copies and schedules
  cudaEvent_t ev_admit = nullptr;  // end of the latest admissions on cst
  DJob *dtab = nullptr, *htab = nullptr;  // 2 lanes x 2 steps x 2 stages x max_slots descriptors
  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0, steps = 0, jobs_in_steps = 0;
  double vox_done = 0;
  bool have_first = false;
  Clock::time_point t_first, t_last;
};

namespace {

size_t srv_job_bytes(const Plan &pl) {
  return al256(pl.g.N * 4) * 2 + al256(2 * sizeof(DJob)) + pl.total;
}

// Descriptor of one job for the stage it runs next.
DJob srv_stage_job(const SrvJob *j, int stage, const bmnd_params &pr) {
  const Plan &pl = j->plan;
  DJob J;
  memset(&J, 0, sizeof(J));
  J.g = pl.g;
  const int stages = j->spec.stages;
  const int M = stage == 1 ? j->spec.group_size[0] : (stages == 2 ? j->spec.group_size[1] : j->spec.group_size[0]);
  fill_stage(J.g, stage, M, j->spec.noise, pr);
  const int mc = j->spec.mass_conserve & (stages == 2 ? 3 : 1);
  const bool m = (mc >> (stage - 1)) & 1;
  unsigned char *B = j->scratch;
  float *pilot = (float *)(B + pl.o_pilot);
  J.y = j->dy;
  J.guide = stage == 1 ? j->dy : pilot;
  J.out = stage == stages ? j->dout : pilot;
  J.eta = m ? (float *)(B + pl.o_eta) : nullptr;
  J.partial = (float2 *)(B + pl.o_partial);
  J.ref_local = (const int *)(B + pl.o_refs);
  J.ref_count = (const int *)(B + pl.o_rcount);
  J.groups = m ? (int *)(B + pl.o_groups) : nullptr;
  J.gcount = m ? (int *)(B + pl.o_gcount) : nullptr;
  if (m && pl.cache) {
    J.pcache = (float *)(B + pl.o_pcache);
    J.wcache = (float *)(B + pl.o_wcache);
    J.ref_base = (const int *)(B + pl.o_refbase);
    J.pcache_refs = pl.cache_refs;
  }
  return J;
}

bmnd_status srv_fail(bmnd_server *S, const char *what, cudaError_t e) {
  snprintf(S->ctx->err, sizeof(S->ctx->err), "%s: %s", what, cudaGetErrorString(e));
  return BMND_ECUDA;
}

// Host callback at the end of a step (no CUDA calls here).
void CUDART_CB srv_step_done(void *p) {
  SrvStepRef *r = static_cast<SrvStepRef *>(p);
  {
    std::lock_guard<std::mutex> lk(r->S->mu);
    r->S->lanes[r->lane].steps[r->slot].done = true;
  }
  r->S->cv_work.notify_all();
}

// One step of a lane, launched asynchronously: every job of T.jobs runs all
// its stages (stage 1, then stage 2 on the pilot), so it completes in this
// step; jobs sharing a kernel class (axes, patch side, candidates per lane)
// share one launch of each kernel per stage.  The lane's stream first waits
// for the latest admissions.
bmnd_status srv_step(bmnd_server *S, SrvLane &L, SrvStep &T) {
  bmnd_params pr;
  bmnd_default_params(&pr);
  cudaError_t e = cudaStreamWaitEvent(L.st, S->ev_admit, 0);
  if (e != cudaSuccess) return srv_fail(S, "admission wait", e);
  for (int stage = 1; stage <= 2; ++stage) {
    std::map<std::pair<int, int>, std::vector<SrvJob *>> classes;
    for (SrvJob *j : T.jobs)
      if (stage <= j->spec.stages) classes[{j->plan.D, kernel_jl(j->plan) * 16 + pick_kb(j->plan)}].push_back(j);
    size_t tab_off = T.tab_base + (size_t)(stage - 1) * S->max_slots;
    for (auto &kv : classes) {
      std::vector<SrvJob *> &cj = kv.second;
      const int D = kv.first.first, jL = kv.first.second / 16, kb = kv.first.second % 16;
      int tiles = 0, smax = 0, smax2 = 0;
      int64_t vox = 0;
      bool any_mc = false;
      for (size_t i = 0; i < cj.size(); ++i) {
        SrvJob *j = cj[i];
        DJob J = srv_stage_job(j, stage, pr);
        J.tile_base = tiles;
        J.vox_base = vox;
        tiles += j->plan.g.ntiles;
        vox += j->plan.g.N;
        const bool m = J.groups != nullptr;
        any_mc = any_mc || m;
        smax = std::max(smax, m ? std::max(j->plan.smem[stage - 1], j->plan.smem[2]) : j->plan.smem[stage - 1]);
        if (m)
          smax2 = std::max(smax2, j->plan.cache ? j->plan.smem_cached
                                                : std::max(j->plan.smem[stage - 1], j->plan.smem[2]));
        S->htab[tab_off + i] = J;
      }
      DJob *dj = S->dtab + tab_off;
      e = cudaMemcpyAsync(dj, S->htab + tab_off, cj.size() * sizeof(DJob), cudaMemcpyHostToDevice, L.st);
      if (e != cudaSuccess) return srv_fail(S, "job table copy", e);
      const int rgrid = (int)std::min<int64_t>((vox + 255) / 256, 148 * 32);
      bmnd_status rc = launch_stage(S->ctx, D, jL, kb, stage, dj, (int)cj.size(), tiles, 0, smax, L.st, L.counter,
                                    L.tile_ctas);
      if (rc != BMND_OK) return rc;
      launch_reduce(D, dj, (int)cj.size(), vox, any_mc ? 1 : 0, rgrid, L.st);
      if (any_mc) {
        rc = launch_stage(S->ctx, D, jL, kb, stage, dj, (int)cj.size(), tiles, 2, smax2, L.st, L.counter,
                          L.tile_ctas);
        if (rc != BMND_OK) return rc;
        launch_reduce(D, dj, (int)cj.size(), vox, 0, rgrid, L.st);
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) return srv_fail(S, "stage launch", e);
      tab_off += cj.size();
    }
  }
  e = cudaLaunchHostFunc(L.st, srv_step_done, &T.ref);
  if (e != cudaSuccess) return srv_fail(S, "step callback", e);
  return BMND_OK;
}

// Admission set-up of one job on the copy stream: input copy, descriptor,
// reference schedule.
bmnd_status srv_admit(bmnd_server *S, SrvJob *j) {
  const Plan &pl = j->plan;
  unsigned char *base = S->arena + j->off;
  const size_t nb = al256(pl.g.N * 4);
  j->dy = (float *)base;
  j->dout = (float *)(base + nb);
  j->djob = (DJob *)(base + 2 * nb);
  j->scratch = base + 2 * nb + al256(2 * sizeof(DJob));
  bmnd_params pr;
  bmnd_default_params(&pr);
  DJob J = srv_stage_job(j, 1, pr);
  cudaError_t e = cudaMemcpyAsync(j->dy, j->spec.y, pl.g.N * 4, cudaMemcpyHostToDevice, S->cst);
  if (e == cudaSuccess) e = cudaMemcpyAsync(j->djob, &J, sizeof(DJob), cudaMemcpyHostToDevice, S->cst);
  if (e == cudaSuccess) e = cudaMemsetAsync(j->scratch + pl.o_flags, 0, (size_t)pl.nflags, S->cst);
  if (e != cudaSuccess) return srv_fail(S, "admission copy", e);
  launch_sched(pl.s, j->scratch + pl.o_flags, j->djob, pl.g.ntiles, (int *)(j->scratch + pl.o_refs),
               (int *)(j->scratch + pl.o_rcount), S->cst);
  if (pl.cache)
    launch_ref_base((const int *)(j->scratch + pl.o_rcount), pl.g.ntiles, (int *)(j->scratch + pl.o_refbase), S->cst);
  e = cudaGetLastError();
  if (e != cudaSuccess) return srv_fail(S, "schedule launch", e);
  return BMND_OK;
}

void srv_finish(bmnd_server *S, SrvJob *j, bmnd_status rc) {
  // caller holds S->mu
  j->status = rc;
  j->state = rc == BMND_OK ? SJ_DONE : SJ_FAILED;
  j->t_done = Clock::now();
  S->alloc.release(j->off, j->bytes);
  S->admit_blocked = false;  // memory and a slot came free
  if (rc == BMND_OK) {
    ++S->completed;
    S->lat_ms.push_back(std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count());
    S->vox_done += (double)j->plan.g.N;
    S->t_last = j->t_done;
  } else {
    ++S->failed;
  }
}

// Estimated milliseconds of a job on one B300 (both stages): candidate
// comparisons x patch entries, at a per-rank rate measured on the paper's
// configurations.  It only chooses the lane.
double srv_job_ms(const Plan &pl, int stages) {
  double cand = 1.0;
  for (int a = 0; a < pl.D; ++a) cand *= 2.0 * pl.g.rad[a] + 1.0;
  const double units = (double)pl.s.nslots * pl.s.passes * cand * pl.g.P * stages;
  const double ms_per_g = pl.D == 1 ? 1.5 : (pl.D == 2 ? 0.55 : 1.0);
  return units * 1e-9 * ms_per_g;
}

// Jobs estimated above this run in the large-job lane.
constexpr double kLargeJobMs = 1.0;

// The worker: completes finished lane steps (results back to the host),
// admits pending jobs in arrival order within the memory budget, and starts
// the next step of every idle lane that has jobs.  Small and large jobs run
// in separate lanes, so a large job's stage (one CTA per tile, low priority)
// never holds back the small jobs' steps by more than a tile.  CUDA calls are
// made without holding the lock.
void srv_loop(bmnd_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  auto waiting = [&](const SrvLane &L) {
    for (const SrvJob *j : L.active)
      if (!j->in_step) return true;
    return false;
  };
  auto lane_ready = [&](const SrvLane &L) {
    bool free_slot = false;
    for (const SrvStep &T : L.steps) {
      if (T.busy && T.done) return true;
      free_slot = free_slot || !T.busy;
    }
    return free_slot && waiting(L);
  };
  for (;;) {
    S->cv_work.wait(lk, [&] {
      return S->stop || (!S->pending.empty() && !S->admit_blocked) || lane_ready(S->lanes[0]) ||
             lane_ready(S->lanes[1]);
    });
    bool idle = true;
    for (const SrvLane &L : S->lanes) idle = idle && L.active.empty() && !L.steps[0].busy && !L.steps[1].busy;
    if (S->stop && S->pending.empty() && idle) break;
    // ---- finished steps
    for (int li = 0; li < 2; ++li) {
      SrvLane &L = S->lanes[li];
      for (SrvStep &T : L.steps) {
        if (!(T.busy && T.done)) continue;
        std::vector<SrvJob *> run;
        run.swap(T.jobs);
        bmnd_status rc = T.rc;
        lk.unlock();
        if (rc == BMND_OK) {
          cudaError_t e = cudaStreamQuery(L.st);
          if (e != cudaSuccess && e != cudaErrorNotReady) rc = srv_fail(S, "step", e);
        }
        for (SrvJob *j : run) {
          if (rc != BMND_OK) continue;
          // pageable destination: the copy has completed when this returns
          cudaError_t e = cudaMemcpyAsync(j->spec.out, j->dout, j->plan.g.N * 4, cudaMemcpyDeviceToHost, S->cst);
          if (e == cudaSuccess) e = cudaStreamSynchronize(S->cst);
          if (e != cudaSuccess) {
            cudaGetLastError();
            j->status = BMND_ECUDA;
          }
        }
        lk.lock();
        T.busy = T.done = false;
        ++S->steps;
        S->jobs_in_steps += (int64_t)run.size();
        for (SrvJob *j : run) {
          L.active.erase(std::find(L.active.begin(), L.active.end(), j));
          srv_finish(S, j, rc != BMND_OK ? rc : j->status);
        }
        S->cv_done.notify_all();
      }
    }
    // ---- admission in arrival order within the memory budget
    std::vector<SrvJob *> admit;
    while (!S->pending.empty()) {
      if ((int)(S->lanes[0].active.size() + S->lanes[1].active.size() + admit.size()) >= S->max_slots) {
        S->admit_blocked = true;
        break;
      }
      SrvJob *j = S->pending.front();
      size_t off = 0;
      if (!S->alloc.alloc(j->bytes, off)) {
        S->admit_blocked = true;
        break;
      }
      j->off = off;
      S->pending.pop_front();
      admit.push_back(j);
    }
    if (!admit.empty()) {
      lk.unlock();
      bmnd_status rc = BMND_OK;
      for (SrvJob *j : admit)
        if (rc == BMND_OK) rc = srv_admit(S, j);
      if (rc == BMND_OK) {
        cudaError_t e = cudaEventRecord(S->ev_admit, S->cst);
        if (e != cudaSuccess) rc = srv_fail(S, "admission event", e);
      }
      if (rc != BMND_OK) cudaStreamSynchronize(S->cst);
      lk.lock();
      for (SrvJob *j : admit) {
        if (rc != BMND_OK) {
          srv_finish(S, j, rc);
          continue;
        }
        j->state = SJ_STAGE1;
        S->lanes[j->lane].active.push_back(j);
      }
      if (rc != BMND_OK) S->cv_done.notify_all();
    }
    // ---- next steps: every free step slot of a lane with waiting jobs
    for (int li = 0; li < 2; ++li) {
      SrvLane &L = S->lanes[li];
      for (SrvStep &T : L.steps) {
        if (T.busy || !waiting(L)) continue;
        T.jobs.clear();
        if (li == 0) {
          // small jobs: all waiting ones, batched
          for (SrvJob *j : L.active)
            if (!j->in_step) T.jobs.push_back(j);
        } else {
          // larger jobs: one per step, the shortest estimate first, aged by
          // the time waited so that none starves
          const Clock::time_point now = Clock::now();
          SrvJob *best = nullptr;
          double best_key = 0;
          for (SrvJob *j : L.active) {
            if (j->in_step) continue;
            const double key = j->est_ms - std::chrono::duration<double, std::milli>(now - j->t_submit).count();
            if (!best || key < best_key) {
              best = j;
              best_key = key;
            }
          }
          T.jobs.push_back(best);
        }
        for (SrvJob *j : T.jobs) j->in_step = true;
        T.busy = true;
        T.done = false;
        lk.unlock();
        bmnd_status rc = srv_step(S, L, T);
        if (rc != BMND_OK) cudaStreamSynchronize(L.st);
        lk.lock();
        T.rc = rc;
        if (rc != BMND_OK) T.done = true;  // no callback was queued
      }
    }
  }
}

// Frees a server's device and host resources (the worker has stopped).
void srv_release(bmnd_server *S) {
  for (int li = 0; li < 2; ++li) {
    if (S->lanes[li].st) cudaStreamDestroy(S->lanes[li].st);
    if (S->lanes[li].counter) cudaFree(S->lanes[li].counter);
  }
  if (S->ev_admit) cudaEventDestroy(S->ev_admit);
  if (S->cst) cudaStreamDestroy(S->cst);
  if (S->arena) cudaFree(S->arena);
  if (S->dtab) cudaFree(S->dtab);
  if (S->htab) cudaFreeHost(S->htab);
  if (S->ctx) bmnd_destroy(S->ctx);
  delete S;
}

}  // namespace

extern "C" {

bmnd_status bmnd_server_create(bmnd_server **out, int device, const bmnd_server_config *cfg) {
  if (!out) return BMND_EINVAL;
  *out = nullptr;
  bmnd_server *S = new bmnd_server();
  S->device = device;
  S->budget = cfg && cfg->mem_budget_bytes ? cfg->mem_budget_bytes : ((size_t)8 << 30);
  S->max_slots = cfg && cfg->max_slots > 0 ? cfg->max_slots : 256;
  bmnd_status rc = bmnd_create(&S->ctx, device, 0);
  if (rc == BMND_OK) {
    cudaSetDevice(device);
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaMalloc(&S->arena, S->budget) != cudaSuccess ||
        cudaMalloc(&S->dtab, sizeof(DJob) * 8 * S->max_slots) != cudaSuccess ||
        cudaMallocHost(&S->htab, sizeof(DJob) * 8 * S->max_slots) != cudaSuccess ||
        cudaMalloc(&S->lanes[0].counter, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&S->lanes[1].counter, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      rc = BMND_ENOMEM;
    } else if (cudaStreamCreateWithPriority(&S->lanes[0].st, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
               cudaStreamCreateWithPriority(&S->lanes[1].st, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
               cudaStreamCreateWithFlags(&S->cst, cudaStreamNonBlocking) != cudaSuccess ||
               cudaEventCreateWithFlags(&S->ev_admit, cudaEventDisableTiming) != cudaSuccess ||
               cudaEventRecord(S->ev_admit, S->cst) != cudaSuccess) {
      rc = BMND_ECUDA;
    }
    for (int li = 0; li < 2; ++li)
      for (int k = 0; k < 2; ++k) {
        S->lanes[li].steps[k].tab_base = (li * 2 + k) * 2 * S->max_slots;
        S->lanes[li].steps[k].ref = SrvStepRef{S, li, k};
      }
    // the large-job lane launches one CTA per tile: the small-job lane's
    // higher-priority CTAs take SMs as the large job's tiles finish
    S->lanes[1].tile_ctas = true;
  }
  if (rc != BMND_OK) {
    srv_release(S);
    return rc;
  }
  S->alloc.init(S->budget);
  S->worker = std::thread(srv_loop, S);
  *out = S;
  return BMND_OK;
}

bmnd_status bmnd_server_submit(bmnd_server *S, const bmnd_job *job, int64_t *ticket) {
  if (!S || !job || !ticket) return BMND_EINVAL;
  if (!job->y || !job->out) return fail(S->ctx, BMND_EINVAL, "null y or out");
  SrvJob *j = new SrvJob();
  j->spec = *job;
  bmnd_params pr;
  bmnd_default_params(&pr);
  bmnd_status rc;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    rc = check_noise(S->ctx, job->noise);
    if (rc == BMND_OK && (job->mass_conserve < 0 || job->mass_conserve > 3))
      rc = fail(S->ctx, BMND_EINVAL, "mass_conserve must be in [0, 3]");
    if (rc == BMND_OK)
      rc = make_plan(S->ctx, job->ndim, job->shape, job->patch, job->step, job->search, job->group_size, job->stages,
                     job->mass_conserve, pr, j->plan);
    if (rc == BMND_OK) {
      // the synthesis cache of mass-conserving jobs, when it takes at most a
      // quarter of the server's budget
      if (job->mass_conserve) {
        add_mc_cache(j->plan);
        if (al256(srv_job_bytes(j->plan)) > S->budget / 4) drop_mc_cache(j->plan);
      }
      j->bytes = al256(srv_job_bytes(j->plan));
      j->est_ms = srv_job_ms(j->plan, job->stages);
      j->lane = j->est_ms > kLargeJobMs ? 1 : 0;
      if (j->bytes > S->budget)
        rc = fail(S->ctx, BMND_ENOMEM, "job needs %zu bytes, the server budget is %zu", j->bytes, S->budget);
    }
    if (rc != BMND_OK) {
      delete j;
      return rc;
    }
    j->ticket = S->next_ticket++;
    j->t_submit = Clock::now();
    if (!S->have_first) {
      S->have_first = true;
      S->t_first = j->t_submit;
    }
    ++S->submitted;
    S->jobs[j->ticket] = j;
    if (S->pending.empty()) S->admit_blocked = false;
    S->pending.push_back(j);
    *ticket = j->ticket;
  }
  S->cv_work.notify_one();
  return BMND_OK;
}

bmnd_status bmnd_server_wait(bmnd_server *S, int64_t ticket, int timeout_ms, double *latency_ms) {
  if (!S) return BMND_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return BMND_EINVAL;
  SrvJob *j = it->second;
  auto done = [&] { return j->state == SJ_DONE || j->state == SJ_FAILED; };
  if (timeout_ms < 0) S->cv_done.wait(lk, done);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) return BMND_ETIMEOUT;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_submit).count();
  bmnd_status rc = j->status;
  S->jobs.erase(it);
  delete j;
  return rc;
}

bmnd_status bmnd_server_get_stats(bmnd_server *S, bmnd_server_stats *o) {
  if (!S || !o) return BMND_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  memset(o, 0, sizeof(*o));
  o->submitted = S->submitted;
  o->completed = S->completed;
  o->failed = S->failed;
  o->steps = S->steps;
  o->mean_jobs_per_step = S->steps ? (double)S->jobs_in_steps / S->steps : 0.0;
  std::vector<double> l = S->lat_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)std::floor(f * (l.size() - 1) + 0.5))]; };
    o->p50_ms = q(0.50);
    o->p99_ms = q(0.99);
    double s = 0;
    for (double v : l) s += v;
    o->mean_ms = s / l.size();
    double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
    o->voxels_per_s = span > 0 ? S->vox_done / span : 0.0;
  }
  return BMND_OK;
}

bmnd_status bmnd_server_destroy(bmnd_server *S) {
  if (!S) return BMND_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto &kv : S->jobs) delete kv.second;
  cudaSetDevice(S->device);
  cudaDeviceSynchronize();
  srv_release(S);
  return BMND_OK;
}

}  // extern "C"
