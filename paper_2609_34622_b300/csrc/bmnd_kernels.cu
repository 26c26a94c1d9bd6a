// Kernels of the B300 BMND denoiser.  See bmnd_kernels.cuh for the work
// decomposition.  Every kernel here is launched from bmnd.cu.
#include "bmnd_kernels.cuh"

#include <float.h>
#include <limits.h>

namespace bmnd {

__constant__ float c_dct[2 * DCT_TOTAL];

cudaError_t upload_dct_constants(const float *h) {
  return cudaMemcpyToSymbol(c_dct, h, sizeof(float) * 2 * DCT_TOTAL);
}

// ---------------------------------------------------------------------------
// reference schedule (Sec. 4.1)
// ---------------------------------------------------------------------------

// Eq. (number-shifts) and Eq. (candidate-shift-list): n_d rounded, uniformly
// spaced shifts in [0, j_d - 1].
__device__ int shift_count(int j, int h, double rho) {
  double v = ceil(rho * (double)(j - 1) / (double)h);
  int n = v < 1.0 ? 1 : (int)v;
  return n < j ? n : j;
}
__device__ int shift_at(int j, int n, int i) {
  if (n == 1) return 0;
  // floor(i (j-1) / (n-1) + 1/2) in exact integer arithmetic
  return (2 * i * (j - 1) + (n - 1)) / (2 * (n - 1));
}

// One thread per (slot tuple, pass): the clipped origin of
// Def. "Clipped reference origin" with offsets of the selected schedule
// (generated / off / sparse / balanced), marked in a byte grid over all
// valid origins.  Duplicates mark the same byte, which deduplicates them.
__global__ void k_sched_mark(SGeom s, unsigned char *__restrict__ flags) {
  int64_t total = s.nslots * (int64_t)s.passes;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(t % s.passes);
    int64_t slot = t / s.passes;
    int64_t q[8];
    int64_t Q = 0;
    for (int d = s.ndim - 1; d >= 0; --d) { q[d] = slot % s.Z[d]; slot /= s.Z[d]; }
    for (int d = 0; d < s.ndim; ++d) Q += q[d];
    int64_t idx = 0;
    for (int d = 0; d < s.ndim; ++d) {
      int n = shift_count(s.j[d], s.h[d], s.rho);
      int64_t o = 0;
      if (s.schedule == 0) {
        if (d < s.ndim - 1) o = shift_at(s.j[d], n, (int)((q[d + 1] + k) % n));
      } else if (s.schedule == 2) {
        bool act = s.Z[d] > 1 || s.j[d] > 1;
        int e = -1;
        for (int a = d + 1; a < s.ndim; ++a)
          if (s.Z[a] > 1 || s.j[a] > 1) { e = a; break; }
        if (act && e >= 0) o = shift_at(s.j[d], n, (int)((q[e] + k) % n));
      } else if (s.schedule == 3) {
        o = shift_at(s.j[d], n, (int)((k + Q - q[d]) % n));
      }
      int64_t nominal = q[d] * s.h[d];
      if (nominal > s.ell[d]) nominal = s.ell[d];
      int64_t r = nominal - o;
      if (r < 0) r = 0;
      if (r > s.ell[d]) r = s.ell[d];
      if (q[d] == s.Z[d] - 1) r = s.ell[d];
      if (s.kax[d] >= 0) idx += r * s.fst[s.kax[d]];
    }
    flags[idx] = 1;
  }
}

// One CTA per tile: compacts the marked origins of the tile's core box, in
// C order, into the tile's reference list.
__global__ void k_sched_compact(const DJob *__restrict__ jobs, int njobs, SGeom s,
                                const unsigned char *__restrict__ flags, int *ref_local,
                                int *ref_count) {
  const DGeom &g = jobs[0].g;
  int tile = blockIdx.x;
  int tc[KMAXD];
  {
    int rem = tile;
    for (int d = g.D - 1; d >= 0; --d) { tc[d] = rem % g.NT[d]; rem /= g.NT[d]; }
  }
  __shared__ int warp_tot[32];
  __shared__ int base_s;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c0 = 0; c0 < g.cap; c0 += blockDim.x) {
    int i = c0 + threadIdx.x;
    int f = 0;
    if (i < g.cap) {
      int rem = i;
      int64_t idx = 0;
      bool ok = true;
      for (int d = g.D - 1; d >= 0; --d) {
        int cc = rem % g.C[d];
        rem /= g.C[d];
        int64_t r = (int64_t)tc[d] * g.C[d] + cc;
        if (r > g.ell[d]) ok = false;
        idx += r * s.fst[d];
      }
      f = ok && flags[idx];
    }
    unsigned b = __ballot_sync(0xffffffffu, f);
    int pre = __popc(b & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[wid] = __popc(b);
    __syncthreads();
    int off = base_s;
    for (int w = 0; w < wid; ++w) off += warp_tot[w];
    if (f) ref_local[(int64_t)tile * g.cap + off + pre] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
      int t = 0;
      for (int w = 0; w < nwarp; ++w) t += warp_tot[w];
      base_s += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) ref_count[tile] = base_s;
}

// ---------------------------------------------------------------------------
// warp-level helpers
// ---------------------------------------------------------------------------

struct KV { float k; int i; };

__device__ __forceinline__ bool kv_less(float ak, int ai, float bk, int bi) {
  return ak < bk || (ak == bk && ai < bi);
}

// Sort one (key, index) pair per lane ascending across the warp (bitonic).
__device__ __forceinline__ void warp_sort(float &k, int &i, int lane) {
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      float ok = __shfl_xor_sync(0xffffffffu, k, stride);
      int oi = __shfl_xor_sync(0xffffffffu, i, stride);
      bool up = (lane & size) == 0;
      bool lower = (lane & stride) == 0;
      bool keep_min = (lower == up);
      bool o_less = kv_less(ok, oi, k, i);
      if (keep_min == o_less) { k = ok; i = oi; }
    }
  }
}

// Merge a sorted warp list (lk, li) with sorted offers (ok, oi): keeps the 32
// smallest of the 64, sorted ascending.
__device__ __forceinline__ void warp_merge(float &lk, int &li, float ok, int oi, int lane) {
  float rk = __shfl_sync(0xffffffffu, ok, 31 - lane);
  int ri = __shfl_sync(0xffffffffu, oi, 31 - lane);
  if (kv_less(rk, ri, lk, li)) { lk = rk; li = ri; }
#pragma unroll
  for (int stride = 16; stride > 0; stride >>= 1) {
    float pk = __shfl_xor_sync(0xffffffffu, lk, stride);
    int pi = __shfl_xor_sync(0xffffffffu, li, stride);
    bool lower = (lane & stride) == 0;
    bool p_less = kv_less(pk, pi, lk, li);
    if (lower == p_less) { lk = pk; li = pi; }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// ---------------------------------------------------------------------------
// 1-D transforms on shared-memory lines
// ---------------------------------------------------------------------------

// Orthonormal DCT-II of a line of length J held in registers.  MODE 0: C x,
// 1: C^T x (inverse), 2: (C.^2) x.
template <int J, int MODE>
__device__ __forceinline__ void dct_line(float *__restrict__ buf, int base, int stride) {
  float x[J];
#pragma unroll
  for (int i = 0; i < J; ++i) x[i] = buf[base + i * stride];
#pragma unroll
  for (int k = 0; k < J; ++k) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < J; ++i) {
      float c = MODE == 0 ? c_dct[dct_off(J) + k * J + i]
              : MODE == 1 ? c_dct[dct_off(J) + i * J + k]
                          : c_dct[DCT_TOTAL + dct_off(J) + k * J + i];
      s = fmaf(c, x[i], s);
    }
    buf[base + k * stride] = s;
  }
}

// Any length J <= 32, matrices from global memory (generic fallback).
// tab: forward matrices of all sizes 1..32 at offset (J-1)J(2J-1)/6, then the
// entrywise squares at +GEN_TOTAL.
__device__ __forceinline__ int gen_off(int J) { return (J - 1) * J * (2 * J - 1) / 6; }

__device__ __noinline__ void dct_line_generic(float *__restrict__ buf, int base, int stride, int J, int mode,
                                 const float *__restrict__ tab) {
  float x[JMAX];
  for (int i = 0; i < J; ++i) x[i] = buf[base + i * stride];
  const float *Mt = tab + (mode == 2 ? GEN_TOTAL : 0) + gen_off(J);
  for (int k = 0; k < J; ++k) {
    float s = 0.f;
    for (int i = 0; i < J; ++i) s = fmaf(mode == 1 ? __ldg(Mt + i * J + k) : __ldg(Mt + k * J + i), x[i], s);
    buf[base + k * stride] = s;
  }
}

// Full-depth orthonormal Haar of length N (power of two) in registers.
// Forward output order: [scaling, coarsest detail, ..., finest details].
// MODE 0 forward, 1 inverse, 2 forward with squared coefficients.
template <int N, int MODE>
__device__ __forceinline__ void haar_line(float *__restrict__ buf, int base, int stride) {
  float x[N], t[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = buf[base + i * stride];
  const float R = 0.70710678118654752f;
  if (MODE != 1) {
#pragma unroll
    for (int len = N; len >= 2; len >>= 1) {
#pragma unroll
      for (int i = 0; i < len / 2; ++i) {
        float a = x[2 * i], b = x[2 * i + 1];
        if (MODE == 2) { t[i] = 0.5f * (a + b); t[len / 2 + i] = 0.5f * (a + b); }
        else { t[i] = R * (a + b); t[len / 2 + i] = R * (a - b); }
      }
#pragma unroll
      for (int i = 0; i < len; ++i) x[i] = t[i];
    }
  } else {
#pragma unroll
    for (int len = 2; len <= N; len <<= 1) {
#pragma unroll
      for (int i = 0; i < len / 2; ++i) {
        float a = x[i], d = x[len / 2 + i];
        t[2 * i] = R * (a + d);
        t[2 * i + 1] = R * (a - d);
      }
#pragma unroll
      for (int i = 0; i < len; ++i) x[i] = t[i];
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) buf[base + i * stride] = x[i];
}

__device__ __noinline__ void spatial_line(float *buf, int base, int stride, int J, int mode,
                                          const float *tab) {
#define BMND_DCT_CASE(JJ)                                                  \
  case JJ:                                                                 \
    if (mode == 0) dct_line<JJ, 0>(buf, base, stride);                     \
    else if (mode == 1) dct_line<JJ, 1>(buf, base, stride);                \
    else dct_line<JJ, 2>(buf, base, stride);                               \
    break;
  switch (J) {
    BMND_DCT_CASE(1) BMND_DCT_CASE(2) BMND_DCT_CASE(3) BMND_DCT_CASE(4) BMND_DCT_CASE(5)
    BMND_DCT_CASE(6) BMND_DCT_CASE(7) BMND_DCT_CASE(8) BMND_DCT_CASE(16) BMND_DCT_CASE(32)
    default: dct_line_generic(buf, base, stride, J, mode, tab);
  }
#undef BMND_DCT_CASE
}

__device__ __noinline__ void member_line(float *buf, int base, int stride, int n, int mode, int gtrans,
                                         const float *tab) {
  if (gtrans == 1) { dct_line_generic(buf, base, stride, n, mode, tab); return; }
#define BMND_HAAR_CASE(NN)                                                 \
  case NN:                                                                 \
    if (mode == 0) haar_line<NN, 0>(buf, base, stride);                    \
    else if (mode == 1) haar_line<NN, 1>(buf, base, stride);               \
    else haar_line<NN, 2>(buf, base, stride);                              \
    break;
  switch (n) {
    BMND_HAAR_CASE(1) BMND_HAAR_CASE(2) BMND_HAAR_CASE(4) BMND_HAAR_CASE(8) BMND_HAAR_CASE(16)
    BMND_HAAR_CASE(32)
    default: break;
  }
#undef BMND_HAAR_CASE
}

// Separable group transform T = (group axis) (x) DCT_j0 (x) ... on a warp's
// shared group buffer of n members.  mode 0: T, 1: T^T = T^{-1}, 2: T.^2.
template <int D>
__device__ void group_xform(float *buf, const DGeom &g, int n, int mode, int lane, const int *vbuf,
                            const float *tab) {
  // spatial axes
#pragma unroll
  for (int a = 0; a < D; ++a) {
    int ja = g.j[a];
    if (ja == 1) continue;
    int per = g.P / ja;  // lines per member along axis a
    int bst_a;           // buffer stride of axis a
    {
      int s = 1;
      if (a < D - 1) {
        s = g.LS;
        for (int e = a + 1; e < D - 1; ++e) s *= g.j[e];
      }
      bst_a = s;
    }
    for (int l = lane; l < n * per; l += 32) {
      int m = l / per, li = l - m * per;
      // li enumerates the coordinates of all axes except a, C order
      int base = m * g.MS;
      int rem = li;
#pragma unroll
      for (int e = D - 1; e >= 0; --e) {
        if (e == a) continue;
        int c = rem % g.j[e];
        rem /= g.j[e];
        int s = 1;
        if (e < D - 1) {
          s = g.LS;
          for (int f = e + 1; f < D - 1; ++f) s *= g.j[f];
        }
        base += c * s;
      }
      spatial_line(buf, base, bst_a, ja, mode, tab);
    }
    __syncwarp();
  }
  // group axis
  if (n > 1) {
    for (int v = lane; v < g.P; v += 32) member_line(buf, vbuf[v], g.MS, n, mode, g.gtrans, tab);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// block matching of one reference (Sec. 4.2 / 4.4, App. A group rules)
// ---------------------------------------------------------------------------

template <int D, int JL, int KB>
__device__ int warp_match(const DGeom &g, const float *__restrict__ S, const int *rr,
                          const int *org, const int *rowoff, int lane, int *mem) {
  int lo[D], W[D];
  int64_t ncand = 1;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int rglob = rr[d] + org[d];
    int l = max(rglob - g.rad[d], 0);
    int h = (int)min((int64_t)rglob + g.rad[d], g.ell[d]);
    lo[d] = l - org[d];
    W[d] = h - l + 1;
    ncand *= W[d];
  }
  int WL = W[D - 1];
  int nchk = (WL + KB - 1) / KB;
  int nouter = (int)(ncand / WL);
  int total = nouter * nchk;
  int rbase = 0, ridx = 0;
  {
    int ws = 1;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      rbase += rr[d] * g.rst[d];
      ridx += (rr[d] - lo[d]) * ws;
      ws *= W[d];
    }
  }
  const float gam = g.gamma, tau = g.tau;
  const float gbias = g.poisson ? 0.f : __fmul_rn(__fmul_rn(2.f, (float)g.P), g.var_g);
  float lk = FLT_MAX;
  int li = INT_MAX;
  float thr = FLT_MAX;
  int thri = INT_MAX;
  int nacc = 0;
  int iters = (total + 31) / 32;
  for (int it = 0; it < iters; ++it) {
    int c = it * 32 + lane;
    float key[KB];
    int idx[KB];
#pragma unroll
    for (int b = 0; b < KB; ++b) { key[b] = FLT_MAX; idx[b] = INT_MAX; }
    if (c < total) {
      int o = c / nchk, kk = c - o * nchk;
      int x0 = kk * KB;
      int kb = min(KB, WL - x0);
      int cbase = lo[D - 1] + x0, widx0 = x0;
      {
        int rem = o, ws = WL;
#pragma unroll
        for (int d = D - 2; d >= 0; --d) {
          int oc = rem % W[d];
          rem /= W[d];
          cbase += (lo[d] + oc) * g.rst[d];
          widx0 += oc * ws;
          ws *= W[d];
        }
      }
      float acc[KB], bs[KB];
#pragma unroll
      for (int b = 0; b < KB; ++b) { acc[b] = 0.f; bs[b] = 0.f; }
      const int jl = JL > 0 ? JL : g.jL;
      for (int r = 0; r < g.rows; ++r) {
        const float *prow = S + rbase + rowoff[r];
        const float *qrow = S + cbase + rowoff[r];
        if (JL > 0) {
          constexpr int JJ = JL > 0 ? JL : 1;
          float p[JJ], q[KB + JJ - 1];
#pragma unroll
          for (int i = 0; i < JJ; ++i) p[i] = prow[i];
#pragma unroll
          for (int i = 0; i < KB + JJ - 1; ++i) q[i] = qrow[i];
          if (g.bias_on) {
#pragma unroll
            for (int i = 0; i < JJ; ++i)
#pragma unroll
              for (int b = 0; b < KB; ++b) {
                float df = __fsub_rn(q[b + i], p[i]);
                acc[b] = fmaf(df, df, acc[b]);
                bs[b] = __fadd_rn(bs[b], fmaxf(__fadd_rn(p[i], q[b + i]), 0.f));
              }
          } else {
#pragma unroll
            for (int i = 0; i < JJ; ++i)
#pragma unroll
              for (int b = 0; b < KB; ++b) {
                float df = __fsub_rn(q[b + i], p[i]);
                acc[b] = fmaf(df, df, acc[b]);
              }
          }
        } else {
          for (int i = 0; i < jl; ++i) {
            float pv = prow[i];
#pragma unroll
            for (int b = 0; b < KB; ++b) {
              float qv = qrow[i + b];
              float df = __fsub_rn(qv, pv);
              acc[b] = fmaf(df, df, acc[b]);
              if (g.bias_on) bs[b] = __fadd_rn(bs[b], fmaxf(__fadd_rn(pv, qv), 0.f));
            }
          }
        }
      }
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        bool ok = b < kb && (widx0 + b) != ridx;
        // rounded exactly as written: no contraction of gam * B into the subtraction
        float B = g.poisson ? __fmul_rn(g.s_p, bs[b]) : gbias;
        float sc = gam > 0.f ? __fsub_rn(acc[b], __fmul_rn(gam, B)) : acc[b];
        if (ok) {
          key[b] = sc;
          idx[b] = widx0 + b;
          nacc += sc < tau;
        }
      }
    }
    // merge this round's candidates into the running best list
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      bool offer = kv_less(key[b], idx[b], thr, thri);
      if (__any_sync(0xffffffffu, offer)) {
        float ok = offer ? key[b] : FLT_MAX;
        int oi = offer ? idx[b] : INT_MAX;
        warp_sort(ok, oi, lane);
        warp_merge(lk, li, ok, oi, lane);
        thr = __shfl_sync(0xffffffffu, lk, g.M - 2 >= 0 ? g.M - 2 : 0);
        thri = __shfl_sync(0xffffffffu, li, g.M - 2 >= 0 ? g.M - 2 : 0);
      }
    }
  }
  nacc = warp_sum_i(nacc);
  int K = g.M - 1;
  int navail = (int)ncand - 1;
  int take = min(nacc, K);
  if (1 + take < g.min_group) take = min(min(g.min_group - 1, K), navail);
  int count = 1 + take;
  if (g.gtrans == 0) {
    int pw = 1;
    while (pw * 2 <= count) pw *= 2;
    count = pw;
  }
  if (lane == 0) mem[0] = rbase;
  if (lane + 1 < count) {
    int rem = li, off = 0;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      int c = rem % W[d];
      rem /= W[d];
      off += (lo[d] + c) * g.rst[d];
    }
    mem[lane + 1] = off;
  }
  __syncwarp();
  return count;
}

// ---------------------------------------------------------------------------
// the stage kernel
// ---------------------------------------------------------------------------

// mode 0: match + filter + aggregate (group tables written if job.groups);
// mode 1: match only, group tables written; mode 2: mass-conservation sweep 2
// (groups read back, corrected patches aggregated with the sweep-1 weights).
template <int D, int JL, int KB>
__global__ void __launch_bounds__(NW * 32, 1)
k_stage(const DJob *__restrict__ jobs, int njobs, int mode, const float *__restrict__ tab) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // locate the job of this tile
  int jb = 0;
  {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].tile_base <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    jb = lo;
  }
  DJob *sj = reinterpret_cast<DJob *>(smem);
  {
    const int *src = reinterpret_cast<const int *>(&jobs[jb]);
    int *dst = reinterpret_cast<int *>(sj);
    for (int i = threadIdx.x; i < (int)(sizeof(DJob) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  // sweep 2 only concerns jobs with mass conservation; the others keep the
  // partials of sweep 1, which the second reduce turns into the same output
  if (mode == 2 && sj->groups == nullptr) return;
  const DGeom &g = sj->g;
  const int tile = blockIdx.x - sj->tile_base;
  const bool stage2 = g.stage == 2;
  const bool mc2 = mode == 2;
  // shared layout
  unsigned char *p = smem + ((sizeof(DJob) + 15) & ~(size_t)15);
  int *vreg = reinterpret_cast<int *>(p); p += sizeof(int) * g.P;
  int *vbuf = reinterpret_cast<int *>(p); p += sizeof(int) * g.P;
  float *omega = reinterpret_cast<float *>(p); p += sizeof(float) * g.P;
  int *rowoff = reinterpret_cast<int *>(p); p += sizeof(int) * g.rows;
  p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
  const int RS = g.region + RPAD;
  float *Sg = reinterpret_cast<float *>(p); p += sizeof(float) * RS;           // guide
  float *Sy = Sg;
  if (stage2) { Sy = reinterpret_cast<float *>(p); p += sizeof(float) * RS; }  // observation
  float *Se = nullptr;
  if (mc2) { Se = reinterpret_cast<float *>(p); p += sizeof(float) * RS; }     // eta
  p = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
  float2 *acc = reinterpret_cast<float2 *>(p); p += sizeof(float2) * g.region;
  int wbytes = (3 * MMAX) * 4 + 2 * g.M * g.MS * 4;
  unsigned char *wp = p + (size_t)warp * wbytes;
  int *mem = reinterpret_cast<int *>(wp);
  float *wts = reinterpret_cast<float *>(wp + MMAX * 4);
  float *rr_s = reinterpret_cast<float *>(wp + 2 * MMAX * 4);
  float *bufA = reinterpret_cast<float *>(wp + 3 * MMAX * 4);
  float *bufB = bufA + g.M * g.MS;

  int tc[D], org[D];
  {
    int rem = tile;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) { tc[d] = rem % g.NT[d]; rem /= g.NT[d]; }
#pragma unroll
    for (int d = 0; d < D; ++d) org[d] = tc[d] * g.C[d] - g.rad[d];
  }
  // tables: region offset, buffer offset and window of every patch entry
  for (int v = threadIdx.x; v < g.P; v += blockDim.x) {
    int rem = v, ro = 0;
    float w = 1.f;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      int c = rem % g.j[d];
      rem /= g.j[d];
      ro += c * g.rst[d];
      w *= g.kaiser[d][c];
    }
    vreg[v] = ro;
    vbuf[v] = (v / g.jL) * g.LS + (v % g.jL);
    omega[v] = w;
    if (v % g.jL == 0) rowoff[v / g.jL] = ro;
  }
  // stage the region(s); locations outside the array are never read as
  // patch entries (candidates are clipped) and are set to zero
  const float *gsrc = sj->guide, *ysrc = sj->y, *esrc = sj->eta;
  for (int e = threadIdx.x; e < RS; e += blockDim.x) {
    float vg = 0.f, vy = 0.f, ve = 0.f;
    if (e < g.region) {
      int rem = e;
      int64_t gi = 0;
      bool in = true;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) {
        int c = rem % g.RG[d];
        rem /= g.RG[d];
        int64_t x = (int64_t)org[d] + c;
        if (x < 0 || x >= g.L[d]) in = false;
        gi += x * g.st[d];
      }
      if (in) {
        vg = __ldg(gsrc + gi);
        if (stage2) vy = __ldg(ysrc + gi);
        if (mc2) ve = __ldg(esrc + gi);
      }
      acc[e] = make_float2(0.f, 0.f);
    }
    Sg[e] = vg;
    if (stage2) Sy[e] = vy;
    if (mc2) Se[e] = ve;
  }
  __syncthreads();

  const int nref = sj->ref_count[tile];
  const int rounds = (nref + NW - 1) / NW;
  const int64_t tslot = (int64_t)tile * g.cap;
  for (int rd = 0; rd < rounds; ++rd) {
    const int ri = rd * NW + warp;
    const bool has = ri < nref;
    int n = 0;
    float alpha = 0.f;
    float *syn = bufB;
    if (has) {
      int rr[D];
      {
        int rem = sj->ref_local[tslot + ri];
#pragma unroll
        for (int d = D - 1; d >= 0; --d) { rr[d] = rem % g.C[d] + g.rad[d]; rem /= g.C[d]; }
      }
      if (!mc2) {
        n = warp_match<D, JL, KB>(g, Sg, rr, org, rowoff, lane, mem);
        if (sj->groups) {
          for (int m = lane; m < g.M; m += 32)
            sj->groups[(tslot + ri) * g.M + m] = m < n ? mem[m] : -1;
          if (lane == 0) sj->gcount[tslot + ri] = n;
        }
      } else {
        n = sj->gcount[tslot + ri];
        for (int m = lane; m < n; m += 32) mem[m] = sj->groups[(tslot + ri) * g.M + m];
        __syncwarp();
      }
      if (mode != 1) {
        const int nP = n * g.P;
        // ---- coefficient variances: sigma_k^2 = sum_i T_ki^2 m_v(u_i) ----
        if (g.poisson) {
          for (int e = lane; e < nP; e += 32) {
            int m = e / g.P, v = e - m * g.P;
            bufA[m * g.MS + vbuf[v]] = g.s_p * fmaxf(Sg[mem[m] + vreg[v]], 0.f);
          }
          __syncwarp();
          group_xform<D>(bufA, g, n, 2, lane, vbuf, tab);
        }
        // ---- forward transform of the guide group (y in stage 1, pilot in stage 2)
        for (int e = lane; e < nP; e += 32) {
          int m = e / g.P, v = e - m * g.P;
          bufB[m * g.MS + vbuf[v]] = Sg[mem[m] + vreg[v]];
        }
        __syncwarp();
        group_xform<D>(bufB, g, n, 0, lane, vbuf, tab);
        // ---- shrinkage; per-coefficient weight terms into bufA ----
        for (int e = lane; e < nP; e += 32) {
          int m = e / g.P, v = e - m * g.P;
          int a = m * g.MS + vbuf[v];
          float s2 = g.poisson ? bufA[a] : g.var_g;
          float X = bufB[a];
          float wterm;
          if (!stage2) {
            // strict inequality with a relative guard of 1e-4: exact ties
            // (common with count data) are zeroed whatever the rounding
            bool keep = fabsf(X) > g.lambda * sqrtf(s2) * 1.0001f;
            bufB[a] = keep ? X : 0.f;
            wterm = keep ? (g.wmodel == 0 ? 1.f : s2) : 0.f;
          } else {
            float S = fmaxf(X * X - g.a_power * s2, 0.f);
            float den = S + g.s_v * s2;
            float G = den > 0.f ? S / den : 0.f;
            bufB[a] = G;
            wterm = g.wmodel == 0 ? G * G : (g.wmodel == 1 ? G * G * s2
                                              : G * G * s2 + (1.f - G) * (1.f - G) * S);
          }
          bufA[a] = wterm;
        }
        __syncwarp();
        // ---- r_l = sum_q (term), per group-axis plane l ----
        for (int m = 0; m < n; ++m) {
          float s = 0.f;
          for (int v = lane; v < g.P; v += 32) s += bufA[m * g.MS + vbuf[v]];
          s = warp_sum(s);
          if (lane == 0) rr_s[m] = s;
        }
        __syncwarp();
        // ---- weights: patch scope R_j = sum_l |V_jl|^2 r_l, group scope sum_l r_l
        if (lane < n) {
          float R = 0.f;
          if (g.wscope == 1) {
            for (int l = 0; l < n; ++l) R += rr_s[l];
          } else if (g.gtrans == 0) {
            R = rr_s[0] / (float)n;
            for (int b = n; b >= 2; b >>= 1) R += rr_s[n / b + lane / b] / (float)b;
          } else {
            const float *Mt = tab + gen_off(n);
            for (int l = 0; l < n; ++l) {
              float c = __ldg(Mt + l * n + lane);
              R += c * c * rr_s[l];
            }
          }
          wts[lane] = R > 0.f ? 1.f / R : 1.f;
        }
        __syncwarp();
        if (stage2) {
          // Wiener: transform the observation group and apply the gains
          for (int e = lane; e < nP; e += 32) {
            int m = e / g.P, v = e - m * g.P;
            bufA[m * g.MS + vbuf[v]] = Sy[mem[m] + vreg[v]];
          }
          __syncwarp();
          group_xform<D>(bufA, g, n, 0, lane, vbuf, tab);
          for (int e = lane; e < nP; e += 32) {
            int m = e / g.P, v = e - m * g.P;
            int a = m * g.MS + vbuf[v];
            bufA[a] *= bufB[a];
          }
          __syncwarp();
          syn = bufA;
        }
        // ---- inverse transform: synthesized patches ----
        group_xform<D>(syn, g, n, 1, lane, vbuf, tab);
        if (mc2) {
          // Def. aggregation-aware constant-synthesis correction: the
          // correction adds alpha = d_g / (zeta^T 1) to every synthesized entry
          float dg = 0.f, z1 = 0.f;
          for (int e = lane; e < nP; e += 32) {
            int m = e / g.P, v = e - m * g.P;
            int u = mem[m] + vreg[v];
            float et = Se[u];
            float z = et > 0.f ? wts[m] * omega[v] / et : 0.f;
            dg = fmaf(z, Sy[u] - syn[m * g.MS + vbuf[v]], dg);
            z1 += z;
          }
          dg = warp_sum(dg);
          z1 = warp_sum(z1);
          alpha = z1 > 0.f ? dg / z1 : 0.f;
        }
      }
    }
    if (mode == 1) continue;
    // ---- ordered, atomic-free accumulation into the tile region ----
    if (!(warp == 0 && rd == 0)) named_sync(1 + warp, 64);
    if (has) {
      for (int m = 0; m < n; ++m) {
        const float wm = wts[m];
        const int base = mem[m];
        for (int v = lane; v < g.P; v += 32) {
          int a = base + vreg[v];
          float wo = wm * omega[v];
          float2 t = acc[a];
          t.x = fmaf(wo, syn[m * g.MS + vbuf[v]] + alpha, t.x);
          t.y += wo;
          acc[a] = t;
        }
        __syncwarp();
      }
    }
    __threadfence_block();
    {
      int nxt = warp + 1 == NW ? 0 : warp + 1;
      if (!(nxt == 0 && rd == rounds - 1)) named_arrive(1 + nxt, 64);
    }
  }
  if (mode == 1) return;
  __syncthreads();
  float2 *dst = sj->partial + (int64_t)tile * g.region;
  for (int e = threadIdx.x; e < g.region; e += blockDim.x) dst[e] = acc[e];
}

// Sum the partials of the tiles covering every location in tile order and
// normalize (Def. "Weighted overlap-add estimate").  Locations without weight
// keep the observation.  If write_eta, the denominator is stored as well.
template <int D>
__global__ void k_reduce(const DJob *__restrict__ jobs, int njobs, int64_t total, int write_eta) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].vox_base <= t) lo = mid; else hi = mid - 1;
    }
    const DJob &J = jobs[lo];
    const DGeom &g = J.g;
    int64_t u = t - J.vox_base;
    int64_t uc[D];
    {
      int64_t rem = u;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) { uc[d] = rem % g.L[d]; rem /= g.L[d]; }
    }
    int tlo[D], thi[D], tcur[D];
    bool any = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int64_t a = uc[d] + g.rad[d] - g.RG[d] + 1;   // t C >= a
      int64_t b = uc[d] + g.rad[d];                 // t C <= b
      int64_t l = a <= 0 ? -((-a) / g.C[d]) : (a + g.C[d] - 1) / g.C[d];
      int64_t h = b / g.C[d];
      if (l < 0) l = 0;
      if (h > g.NT[d] - 1) h = g.NT[d] - 1;
      tlo[d] = (int)l;
      thi[d] = (int)h;
      tcur[d] = (int)l;
      if (l > h) any = false;
    }
    float num = 0.f, den = 0.f;
    while (any) {
      int tile = 0, local = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        tile = tile * g.NT[d] + tcur[d];
        local += (int)(uc[d] - ((int64_t)tcur[d] * g.C[d] - g.rad[d])) * g.rst[d];
      }
      float2 v = J.partial[(int64_t)tile * g.region + local];
      num += v.x;
      den += v.y;
      int d = D - 1;
      while (d >= 0) {
        if (++tcur[d] <= thi[d]) break;
        tcur[d] = tlo[d];
        --d;
      }
      if (d < 0) break;
    }
    J.out[u] = den > 0.f ? num / den : J.y[u];
    if (write_eta && J.eta) J.eta[u] = den;
  }
}

// Convert the group tables (region offsets) of one job to linear origins.
template <int D>
__global__ void k_export_groups(const DJob *__restrict__ jobs, const int64_t *__restrict__ tile_off,
                                int64_t *origins, int64_t *groups, int32_t *counts, int64_t cap) {
  const DJob &J = jobs[0];
  const DGeom &g = J.g;
  int tile = blockIdx.x;
  int tc[D];
  {
    int rem = tile;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) { tc[d] = rem % g.NT[d]; rem /= g.NT[d]; }
  }
  int nref = J.ref_count[tile];
  int64_t base = tile_off[tile];
  for (int i = threadIdx.x; i < nref * g.M; i += blockDim.x) {
    int ri = i / g.M, m = i - ri * g.M;
    int64_t slot = base + ri;
    if (slot >= cap) continue;
    int64_t tslot = (int64_t)tile * g.cap + ri;
    if (m == 0) {
      int rem = J.ref_local[tslot];
      int64_t lin = 0;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) {
        lin += ((int64_t)tc[d] * g.C[d] + rem % g.C[d]) * g.st[d];
        rem /= g.C[d];
      }
      origins[slot] = lin;
      if (counts) counts[slot] = J.gcount ? J.gcount[tslot] : 0;
    }
    if (groups) {
      int n = J.gcount[tslot];
      int64_t lin = -1;
      if (m < n) {
        int rem = J.groups[tslot * g.M + m];
        lin = 0;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
          int c = rem % g.RG[d];
          rem /= g.RG[d];
          lin += ((int64_t)tc[d] * g.C[d] - g.rad[d] + c) * g.st[d];
        }
      }
      groups[slot * g.M + m] = lin;
    }
  }
}

// ---------------------------------------------------------------------------
// explicit instantiations and launch helpers
// ---------------------------------------------------------------------------

typedef void (*stage_fn)(const DJob *, int, int, const float *);

template <int D, int JL, int KB>
stage_fn stage_ptr() { return &k_stage<D, JL, KB>; }

stage_fn select_stage_kernel(int D, int jL, int kb) {
  switch (D) {
    case 1:
      if (jL == 32 && kb == 5) return stage_ptr<1, 32, 5>();
      if (jL == 16 && kb == 4) return stage_ptr<1, 16, 4>();
      return stage_ptr<1, 0, 4>();
    case 2:
      if (jL == 8 && kb == 8) return stage_ptr<2, 8, 8>();
      if (jL == 4 && kb == 4) return stage_ptr<2, 4, 4>();
      return stage_ptr<2, 0, 4>();
    case 3:
      if (jL == 4 && kb == 4) return stage_ptr<3, 4, 4>();
      return stage_ptr<3, 0, 4>();
    case 4: return stage_ptr<4, 0, 4>();
    case 5: return stage_ptr<5, 0, 4>();
    case 6: return stage_ptr<6, 0, 4>();
  }
  return nullptr;
}

void launch_reduce(int D, const DJob *jobs, int njobs, int64_t total, int write_eta, int grid,
                   cudaStream_t st) {
  switch (D) {
    case 1: k_reduce<1><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 2: k_reduce<2><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 3: k_reduce<3><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 4: k_reduce<4><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 5: k_reduce<5><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 6: k_reduce<6><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
  }
}

void launch_export(int D, const DJob *jobs, int ntiles, const int64_t *tile_off, int64_t *origins,
                   int64_t *groups, int32_t *counts, int64_t cap, cudaStream_t st) {
  switch (D) {
    case 1: k_export_groups<1><<<ntiles, 128, 0, st>>>(jobs, tile_off, origins, groups, counts, cap); break;
    case 2: k_export_groups<2><<<ntiles, 128, 0, st>>>(jobs, tile_off, origins, groups, counts, cap); break;
    case 3: k_export_groups<3><<<ntiles, 128, 0, st>>>(jobs, tile_off, origins, groups, counts, cap); break;
    case 4: k_export_groups<4><<<ntiles, 128, 0, st>>>(jobs, tile_off, origins, groups, counts, cap); break;
    case 5: k_export_groups<5><<<ntiles, 128, 0, st>>>(jobs, tile_off, origins, groups, counts, cap); break;
    case 6: k_export_groups<6><<<ntiles, 128, 0, st>>>(jobs, tile_off, origins, groups, counts, cap); break;
  }
}

void launch_sched(const SGeom &s, unsigned char *flags, const DJob *jobs, int ntiles, int *ref_local,
                  int *ref_count, cudaStream_t st) {
  int64_t total = s.nslots * s.passes;
  int grid = (int)((total + 255) / 256);
  if (grid > 148 * 16) grid = 148 * 16;
  if (grid < 1) grid = 1;
  k_sched_mark<<<grid, 256, 0, st>>>(s, flags);
  k_sched_compact<<<ntiles, 256, 0, st>>>(jobs, 1, s, flags, ref_local, ref_count);
}

cudaError_t set_stage_smem(stage_fn f, int bytes) {
  return cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace bmnd
