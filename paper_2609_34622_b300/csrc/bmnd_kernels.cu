// Kernels of the B300 BMND denoiser.  See bmnd_kernels.cuh for the work
// decomposition.  Every kernel here is launched from bmnd.cu.
#include "bmnd_kernels.cuh"

#include <type_traits>

#include <float.h>
#include <limits.h>

namespace bmnd {


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

// Reference coverage (Sec. 9.3): one thread per location x (grid-stride),
// C(x) = sum over the patch offsets o of flag[x - o] over the valid origins
// x - o -- a gather over the schedule's byte grid, so the map needs no
// atomics.  sums[0], sums[1], sums[2] accumulate sum C, sum C^2 and the
// number of scheduled origins with integer atomics (order-independent).
__global__ void k_coverage(CovGeom c, const unsigned char *__restrict__ flags, int32_t *__restrict__ cov,
                           unsigned long long *__restrict__ sums) {
  unsigned long long s1 = 0, s2 = 0, nr = 0;
  const int64_t total = c.N > c.nflags ? c.N : c.nflags;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (t < c.N) {
      int64_t x[KMAXD];
      int64_t rem = t;
      for (int a = c.D - 1; a >= 0; --a) {
        x[a] = rem % c.L[a];
        rem /= c.L[a];
      }
      int cnt = 0;
      for (int i = 0; i < c.P; ++i) {
        int ri = i;
        int64_t idx = 0;
        bool ok = true;
        for (int a = c.D - 1; a >= 0; --a) {
          const int o = ri % c.j[a];
          ri /= c.j[a];
          const int64_t r = x[a] - o;
          ok = ok && r >= 0 && r <= c.ell[a];
          idx += r * c.fst[a];
        }
        if (ok) cnt += flags[idx];
      }
      if (cov) cov[t] = cnt;
      s1 += (unsigned long long)cnt;
      s2 += (unsigned long long)cnt * (unsigned long long)cnt;
    }
    if (t < c.nflags) nr += flags[t];
  }
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, off);
    s2 += __shfl_down_sync(0xffffffffu, s2, off);
    nr += __shfl_down_sync(0xffffffffu, nr, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], s1);
    atomicAdd(&sums[1], s2);
    atomicAdd(&sums[2], nr);
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

// (key, index) pairs order by key, then by index; T is float (FP32
// screening) or double (double-precision decisions).
template <typename T>
__device__ __forceinline__ bool kv_less(T ak, int ai, T bk, int bi) {
  return ak < bk || (ak == bk && ai < bi);
}

// Sort one (key, index) pair per lane ascending across the warp (bitonic).
template <typename T>
__device__ __forceinline__ void warp_sort(T &k, int &i, int lane) {
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      T ok = __shfl_xor_sync(0xffffffffu, k, stride);
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
template <typename T>
__device__ __forceinline__ void warp_merge(T &lk, int &li, T ok, int oi, int lane) {
  T rk = __shfl_sync(0xffffffffu, ok, 31 - lane);
  int ri = __shfl_sync(0xffffffffu, oi, 31 - lane);
  if (kv_less(rk, ri, lk, li)) { lk = rk; li = ri; }
#pragma unroll
  for (int stride = 16; stride > 0; stride >>= 1) {
    T pk = __shfl_xor_sync(0xffffffffu, lk, stride);
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
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// single-instruction warp reductions of 32-bit integers
__device__ __forceinline__ int warp_max_i(int v) { return __reduce_max_sync(0xffffffffu, v); }
__device__ __forceinline__ int warp_sum_i(int v) { return __reduce_add_sync(0xffffffffu, v); }

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// ---------------------------------------------------------------------------
// 1-D transforms on shared-memory lines
// ---------------------------------------------------------------------------

// Any length J <= 32 with the matrix read from global memory (used for the
// optional DCT along the group axis, whose length varies per group).
// tab: forward matrices of all sizes 1..32 at offset (J-1)J(2J-1)/6, then the
// entrywise squares at +GEN_TOTAL.  mode 0: M x, 1: M^T x, 2: (M.^2) x.
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

// The optional DCT along the group axis: every entry's line of n members
// (stride MS) of the warp's group buffer.
__device__ __noinline__ void dct_group_axis(float *buf, int P, int MS, int n, int mode, int lane,
                                            const int *__restrict__ vbuf, const float *__restrict__ tab) {
  for (int v = lane; v < P; v += 32) dct_line_generic(buf, vbuf[v], MS, n, mode, tab);
}

// Dense transform of nlines lines of length J held in a warp's shared group
// buffer: line l starts at base_of(l) with element stride st.  M is a J x J
// row-major matrix in shared memory (forward, transposed-for-inverse or
// squared).  When there are fewer lines than lanes, L lanes share a line and
// split its outputs; every lane first loads its line into registers, then the
// warp synchronizes, then outputs are written in place.
template <int J, typename BaseOf>
__device__ __forceinline__ void xform_lines(float *__restrict__ buf, int nlines, BaseOf base_of, int st,
                                            const float *__restrict__ M, int lane) {
  int L = 1;
  while (L * 2 * nlines <= 32 && L * 2 <= J) L *= 2;
  const int items = nlines * L;
#pragma unroll 1
  for (int i0 = 0; i0 < items; i0 += 32) {
    const int item = i0 + lane;
    const bool act = item < items;
    const int l = act ? item / L : 0, sub = act ? item - (item / L) * L : 0;
    const int base = act ? base_of(l) : 0;
    float x[J];
    if (act) {
#pragma unroll
      for (int i = 0; i < J; ++i) x[i] = buf[base + i * st];
    }
    __syncwarp();
    if (act) {
      for (int k = sub; k < J; k += L) {
        const float *row = M + k * J;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        if constexpr (J % 4 == 0) {
#pragma unroll
          for (int i = 0; i < J / 4; ++i) {
            float4 c = reinterpret_cast<const float4 *>(row)[i];
            s0 = fmaf(c.x, x[4 * i], s0);
            s1 = fmaf(c.y, x[4 * i + 1], s1);
            s2 = fmaf(c.z, x[4 * i + 2], s2);
            s3 = fmaf(c.w, x[4 * i + 3], s3);
          }
        } else {
#pragma unroll
          for (int i = 0; i < J; ++i) s0 = fmaf(row[i], x[i], s0);
        }
        buf[base + k * st] = (s0 + s1) + (s2 + s3);
      }
    }
    __syncwarp();
  }
}

// Full-depth orthonormal Haar of length N (power of two) in registers.
// Forward output order: [scaling, coarsest detail, ..., finest details].
// Levels are unrolled by template recursion so that every index is a
// compile-time constant and the line stays in registers.
template <int N, int LEN, bool SQ>
__device__ __forceinline__ void haar_fwd_levels(float (&x)[N]) {
  if constexpr (LEN >= 2) {
    const float R = 0.70710678118654752f;
    float t[LEN];
#pragma unroll
    for (int i = 0; i < LEN / 2; ++i) {
      const float a = x[2 * i], b = x[2 * i + 1];
      if (SQ) { t[i] = 0.5f * (a + b); t[LEN / 2 + i] = 0.5f * (a + b); }
      else { t[i] = R * (a + b); t[LEN / 2 + i] = R * (a - b); }
    }
#pragma unroll
    for (int i = 0; i < LEN; ++i) x[i] = t[i];
    haar_fwd_levels<N, LEN / 2, SQ>(x);
  }
}

template <int N, int LEN>
__device__ __forceinline__ void haar_inv_levels(float (&x)[N]) {
  if constexpr (LEN <= N) {
    const float R = 0.70710678118654752f;
    float t[LEN];
#pragma unroll
    for (int i = 0; i < LEN / 2; ++i) {
      const float a = x[i], d = x[LEN / 2 + i];
      t[2 * i] = R * (a + d);
      t[2 * i + 1] = R * (a - d);
    }
#pragma unroll
    for (int i = 0; i < LEN; ++i) x[i] = t[i];
    haar_inv_levels<N, LEN * 2>(x);
  }
}

// MODE 0 forward, 1 inverse, 2 forward with squared coefficients.
template <int N, int MODE>
__device__ __forceinline__ void haar_line(float *__restrict__ buf, int base, int stride) {
  float x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = buf[base + i * stride];
  if (MODE == 1) haar_inv_levels<N, 2>(x);
  else haar_fwd_levels<N, N, MODE == 2>(x);
#pragma unroll
  for (int i = 0; i < N; ++i) buf[base + i * stride] = x[i];
}

template <int N>
__device__ __forceinline__ void haar_line_mode(float *buf, int base, int stride, int mode) {
  if (mode == 0) haar_line<N, 0>(buf, base, stride);
  else if (mode == 1) haar_line<N, 1>(buf, base, stride);
  else haar_line<N, 2>(buf, base, stride);
}

// Fast DCT of power-of-two length in registers (B. G. Lee, "A new algorithm
// to compute the discrete cosine transform", IEEE Trans. ASSP 32(6), 1984):
// the even outputs of a length-N DCT-II are a length-N/2 DCT-II of
// x_n + x_{N-1-n}; the odd outputs are X_{2k+1} = Y_k + Y_{k+1}, where Y is a
// length-N/2 DCT-II of (x_n - x_{N-1-n}) / (2 cos(pi (2n+1) / (2N))), because
// cos((2k+1) t) = (cos(2k t) + cos(2(k+1) t)) / (2 cos t).  The DCT-III
// (transpose) follows from the same identity read backwards.
// c_sec holds 1 / (2 cos(pi (2n+1) / (2N))) for N = 2, 4, 8, 16, 32 at offset
// N/2 - 1 + n; c_scale holds sqrt(1/N) and sqrt(2/N) at 2 log2(N) (+1).
__constant__ float c_sec[32];
__constant__ float c_scale[12];

cudaError_t upload_fast_dct_constants(const float *sec31, const float *scale12) {
  cudaError_t e = cudaMemcpyToSymbol(c_sec, sec31, sizeof(float) * 31);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_scale, scale12, sizeof(float) * 12);
}

template <int N>
struct Lee {
  // unnormalized DCT-II, in place: X_k = sum_n x_n cos(pi (2n+1) k / (2N))
  static __device__ __forceinline__ void fwd(float (&x)[N]) {
    float a[N / 2], b[N / 2];
#pragma unroll
    for (int n = 0; n < N / 2; ++n) {
      a[n] = x[n] + x[N - 1 - n];
      b[n] = (x[n] - x[N - 1 - n]) * c_sec[N / 2 - 1 + n];
    }
    Lee<N / 2>::fwd(a);
    Lee<N / 2>::fwd(b);
#pragma unroll
    for (int k = 0; k < N / 2; ++k) x[2 * k] = a[k];
#pragma unroll
    for (int k = 0; k < N / 2 - 1; ++k) x[2 * k + 1] = b[k] + b[k + 1];
    x[N - 1] = b[N / 2 - 1];
  }
  // unnormalized DCT-III, in place: x_n = sum_k X_k cos(pi (2n+1) k / (2N))
  static __device__ __forceinline__ void inv(float (&X)[N]) {
    float e[N / 2], p[N / 2];
#pragma unroll
    for (int k = 0; k < N / 2; ++k) e[k] = X[2 * k];
    p[0] = X[1];
#pragma unroll
    for (int m = 1; m < N / 2; ++m) p[m] = X[2 * m + 1] + X[2 * m - 1];
    Lee<N / 2>::inv(e);
    Lee<N / 2>::inv(p);
#pragma unroll
    for (int n = 0; n < N / 2; ++n) {
      float B = p[n] * c_sec[N / 2 - 1 + n];
      X[n] = e[n] + B;
      X[N - 1 - n] = e[n] - B;
    }
  }
};
template <>
struct Lee<1> {
  static __device__ __forceinline__ void fwd(float (&)[1]) {}
  static __device__ __forceinline__ void inv(float (&)[1]) {}
};

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }
__host__ __device__ constexpr int ipow(int b, int e) { return e <= 0 ? 1 : b * ipow(b, e - 1); }

// Patch shape known at compile time: the specialized kernels take cubic
// patches of side JC on all D axes (JC = 0: the shape is read from the
// geometry at run time).  Patches of up to 32 entries are filtered with the
// members in registers (rf): unpadded rows (LS = JC) and an odd member stride
// MS = P | 1.  Larger ones use the shared-memory line transforms: rows
// padded to an odd stride, unpadded multiples of 4 in lean mode (D >= 3).
// The host lays the group buffers out the same way.
template <int D, int JC>
struct CubeShape {
  static constexpr bool fixed = JC > 0;
  static constexpr int P = fixed ? ipow(JC, D) : 0;
  static constexpr bool rf = fixed && P <= 32;
  static constexpr int LS = !fixed ? 0 : (rf || (D >= 3 && JC % 4 == 0)) ? JC : JC + (JC % 2 == 0 ? 1 : 0);
  static constexpr int MS = !fixed ? 0 : rf ? (P | 1) : ipow(JC, D - 1) * LS;
};

// Orthonormal DCT of a line held in registers (length J, power of two).
// MODE 0: C x; 1: C^T x; 2: (C.^2) x, using
// C_ki^2 = c_k^2 (1 + cos(pi (2i+1) 2k / (2J))) / 2: the squared transform is
// (sum_i m_i + s_k V_r) / J with V a length-J/2 DCT-II of m_i + m_{J-1-i}
// (r = k for 0 < k < J/2 with s_k = +1, r = J - k for k > J/2 with s_k = -1,
// and no V term for k = 0 and k = J/2).
template <int J, int MODE>
__device__ __forceinline__ void dct_reg(float (&x)[J]) {
  const float s0 = c_scale[2 * ilog2c(J)], s1 = c_scale[2 * ilog2c(J) + 1];
  if constexpr (MODE == 0) {
    Lee<J>::fwd(x);
    x[0] *= s0;
#pragma unroll
    for (int k = 1; k < J; ++k) x[k] *= s1;
  } else if constexpr (MODE == 1) {
    x[0] *= s0;
#pragma unroll
    for (int k = 1; k < J; ++k) x[k] *= s1;
    Lee<J>::inv(x);
  } else {
    float S = 0.f;
#pragma unroll
    for (int i = 0; i < J; ++i) S += x[i];
    const float invJ = 1.f / (float)J;
    if constexpr (J >= 2) {
      float a[J / 2];
#pragma unroll
      for (int i = 0; i < J / 2; ++i) a[i] = x[i] + x[J - 1 - i];
      Lee<J / 2>::fwd(a);
      x[0] = S * invJ;
#pragma unroll
      for (int k = 1; k < J / 2; ++k) x[k] = (S + a[k]) * invJ;
      x[J / 2] = S * invJ;
#pragma unroll
      for (int k = J / 2 + 1; k < J; ++k) x[k] = (S - a[J - k]) * invJ;
    } else {
      x[0] = S * invJ;
    }
  }
}

// The same on one line of a shared buffer with stride st (mode 0 / 1 / 2).
template <int J>
__device__ __forceinline__ void fast_dct_line(float *__restrict__ buf, int base, int st, int mode, bool vec4) {
  float x[J];
  // vec4: a stride-1 line of unpadded rows (LS a multiple of 4), which starts
  // on a 16-byte boundary; read and written as float4
  const bool vec = (J % 4 == 0) && vec4;
  if (vec) {
#pragma unroll
    for (int i = 0; i < J; i += 4) {
      const float4 q = *reinterpret_cast<const float4 *>(buf + base + i);
      x[i] = q.x; x[i + 1] = q.y; x[i + 2] = q.z; x[i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < J; ++i) x[i] = buf[base + i * st];
  }
  if (mode == 0) dct_reg<J, 0>(x);
  else if (mode == 1) dct_reg<J, 1>(x);
  else dct_reg<J, 2>(x);
  if (vec) {
#pragma unroll
    for (int i = 0; i < J; i += 4)
      *reinterpret_cast<float4 *>(buf + base + i) = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < J; ++i) buf[base + i * st] = x[i];
  }
}

// Separable DCT (MODE as in dct_reg) of a whole cubic patch of side JC held
// in registers, C-order entries; axes in order 0 .. D-1.
template <int D, int JC, int MODE, int A = 0>
__device__ __forceinline__ void dct_patch(float (&x)[ipow(JC, D)]) {
  if constexpr (A < D) {
    constexpr int S = ipow(JC, D - 1 - A);
    constexpr int P = ipow(JC, D);
#pragma unroll
    for (int l = 0; l < P / JC; ++l) {
      const int base = (l / S) * (S * JC) + (l % S);
      float t[JC];
#pragma unroll
      for (int i = 0; i < JC; ++i) t[i] = x[base + i * S];
      dct_reg<JC, MODE>(t);
#pragma unroll
      for (int i = 0; i < JC; ++i) x[base + i * S] = t[i];
    }
    dct_patch<D, JC, MODE, A + 1>(x);
  }
}

// Shared-memory matrices of one patch axis: [forward F | synthesis S |
// squared F.^2 | F^T]; mode 0..3 selects one (S = F^T for the DCT).
__device__ __forceinline__ const float *axis_matrix(const float *mats, const int *moff, int a, int J, int mode) {
  return mats + moff[a] + mode * J * J;
}

// Separable group transform T = (group axis) (x) F_j0 (x) ... on a warp's
// shared group buffer of n members, F the orthonormal DCT or bior1.5
// (g.spatial).  mode 0: T, 1: the synthesis T^{-1} (T^T for the DCT),
// 2: T.^2.  The DCT runs as register butterflies on power-of-two axes;
// bior1.5 and other lengths as dense products with the shared matrices.
// Dense transform along patch axis a of a compile-time cubic shape (the
// non-orthonormal bior1.5 spatial transform, matrix M in shared memory),
// every line of the n member patches.  Out of line: only arrays with that
// transform take it, and inlined beside the butterflies it costs the stage
// kernels registers.
template <int D, int JC>
__device__ __noinline__ void dense_axis_fixed(float *buf, int n, int a, const float *M, int lane) {
  using SH = CubeShape<D, JC>;
  constexpr int per = SH::P / JC;  // lines per member along any axis
  int bs[D];
  {
    int s = 1;
#pragma unroll
    for (int e = D - 1; e >= 0; --e) {
      if (e == D - 1) { bs[e] = 1; s = SH::LS; }
      else { bs[e] = s; s *= JC; }
    }
  }
  auto base_of = [&](int l) {
    int m = l / per, li = l - m * per;
    int base = m * SH::MS, rem = li;
#pragma unroll
    for (int e = D - 1; e >= 0; --e) {
      if (e == a) continue;
      int c = rem % JC;
      rem /= JC;
      base += c * bs[e];
    }
    return base;
  };
  xform_lines<JC>(buf, n * per, base_of, bs[a], M, lane);
}

template <int D, int JC>
__device__ __forceinline__ void group_xform(float *buf, const DGeom &g, int n, int mode, int lane, const int *vbuf,
                            const float *mats, const int *moff, const float *tab) {
  using SH = CubeShape<D, JC>;
  const int P = SH::fixed ? SH::P : g.P;
  const int LS = SH::fixed ? SH::LS : g.LS;
  const int MS = SH::fixed ? SH::MS : g.MS;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int ja = SH::fixed ? JC : g.j[a];
    if (ja == 1) continue;
    const int per = P / ja;  // lines per member along axis a
    int bs[D];
    {
      int s = 1;
#pragma unroll
      for (int e = D - 1; e >= 0; --e) {
        if (e == D - 1) { bs[e] = 1; s = LS; }
        else { bs[e] = s; s *= SH::fixed ? JC : g.j[e]; }
      }
    }
    auto base_of = [&](int l) {
      int m = l / per, li = l - m * per;
      int base = m * MS, rem = li;
#pragma unroll
      for (int e = D - 1; e >= 0; --e) {
        if (e == a) continue;
        const int je = SH::fixed ? JC : g.j[e];
        int c = rem % je;
        rem /= je;
        base += c * bs[e];
      }
      return base;
    };
    const float *M = axis_matrix(mats, moff, a, ja, mode);
    const int nl = n * per, st = bs[a];
    const bool vec4 = a == D - 1 && (LS & 3) == 0;
    if constexpr (SH::fixed) {
      if (g.spatial) {
        dense_axis_fixed<D, JC>(buf, n, a, M, lane);
        continue;
      }
    }
    if ((ja & (ja - 1)) == 0 && (SH::fixed || !g.spatial)) {
      // power-of-two length: register butterflies, one lane per line
#pragma unroll 1
      for (int l = lane; l < nl; l += 32) {
        const int base = base_of(l);
        switch (ja) {
          case 2: fast_dct_line<2>(buf, base, st, mode, vec4); break;
          case 4: fast_dct_line<4>(buf, base, st, mode, vec4); break;
          case 8: fast_dct_line<8>(buf, base, st, mode, vec4); break;
          case 16: fast_dct_line<16>(buf, base, st, mode, vec4); break;
          default: fast_dct_line<32>(buf, base, st, mode, vec4); break;
        }
      }
      __syncwarp();
      continue;
    }
    switch (ja) {
      case 2: xform_lines<2>(buf, nl, base_of, st, M, lane); break;
      case 3: xform_lines<3>(buf, nl, base_of, st, M, lane); break;
      case 4: xform_lines<4>(buf, nl, base_of, st, M, lane); break;
      case 8: xform_lines<8>(buf, nl, base_of, st, M, lane); break;
      case 16: xform_lines<16>(buf, nl, base_of, st, M, lane); break;
      case 32: xform_lines<32>(buf, nl, base_of, st, M, lane); break;
      case 5: xform_lines<5>(buf, nl, base_of, st, M, lane); break;
      case 6: xform_lines<6>(buf, nl, base_of, st, M, lane); break;
      case 7: xform_lines<7>(buf, nl, base_of, st, M, lane); break;
      case 12: xform_lines<12>(buf, nl, base_of, st, M, lane); break;
      default:
        for (int l = lane; l < nl; l += 32) dct_line_generic(buf, base_of(l), st, ja, mode, tab);
        __syncwarp();
    }
  }
  // group axis
  if (n > 1 && g.gtrans == 1) {
    dct_group_axis(buf, P, MS, n, mode, lane, vbuf, tab);
  } else if (n > 1) {
#pragma unroll 1
    for (int v = lane; v < P; v += 32) {
      const int base = vbuf[v];
      switch (n) {
        case 2: haar_line_mode<2>(buf, base, MS, mode); break;
        case 4: haar_line_mode<4>(buf, base, MS, mode); break;
        case 8: haar_line_mode<8>(buf, base, MS, mode); break;
        case 16: haar_line_mode<16>(buf, base, MS, mode); break;
        case 32: haar_line_mode<32>(buf, base, MS, mode); break;
        default: break;
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Poisson matching distances (Sec. 4.2) and their finite-count calibration
// (Sec. 4.3).  Scores and thresholds are float32 with every operation rounded
// once, in the order written (explicit intrinsics, no contraction), so the
// groups they decide are the same on every run and build.
// ---------------------------------------------------------------------------

// ln x for x > 0 by the artanh series: x = 2^e m with m in [1/sqrt 2, sqrt 2],
// s = (m - 1) / (m + 1) (|s| <= 0.172), ln m = 2 (s + s^3/3 + ... + s^9/9)
// (the omitted terms are below 1e-9 relative), plus e ln 2 with ln 2 split
// into a 16-bit head (e times it is exact) and a float tail.
__device__ __forceinline__ float series_log(float x) {
  int e = 0;
  if (x < FLT_MIN) {
    x = __fmul_rn(x, 0x1p23f);
    e = -23;
  }
  const unsigned b = __float_as_uint(x);
  e += (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.f), __fadd_rn(m, 1.f));
  const float s2 = __fmul_rn(s, s);
  float q = __fmaf_rn(s2, 0x1.c71c72p-3f, 0x1.24924ap-2f);  // 2/9, 2/7
  q = __fmaf_rn(s2, q, 0x1.99999ap-2f);                      // 2/5
  q = __fmaf_rn(s2, q, 0x1.555556p-1f);                      // 2/3
  q = __fmaf_rn(s2, q, 2.f);
  const float lm = __fmul_rn(s, q);
  const float fe = (float)e;
  return __fmaf_rn(fe, 0x1.62e4p-1f, __fmaf_rn(fe, 0x1.7f7d1cp-20f, lm));
}

// Per-entry contribution phi_m(r, c) of Eq. (varphi): 1 Poisson deviance
// (Eq. deviance, 0 log 0 = 0), 2 Pearson (Eq. pearson), 3 half the squared
// Anscombe difference (Eq. anscombe-distance); a zero total contributes 0.
template <int METRIC>
__device__ __forceinline__ float poisson_phi(float r, float c) {
  const float n = __fadd_rn(r, c);
  if (METRIC == 1) {
    if (!(n > 0.f)) return 0.f;
    const float a = r > 0.f ? __fmul_rn(r, series_log(__fdiv_rn(__fmul_rn(2.f, r), n))) : 0.f;
    const float b = c > 0.f ? __fmul_rn(c, series_log(__fdiv_rn(__fmul_rn(2.f, c), n))) : 0.f;
    return __fmul_rn(2.f, __fadd_rn(a, b));
  } else if (METRIC == 2) {
    if (!(n > 0.f)) return 0.f;
    const float d = __fsub_rn(r, c);
    return __fdiv_rn(__fmul_rn(d, d), n);
  } else {
    const float d = __fsub_rn(__fmul_rn(2.f, __fsqrt_rn(__fadd_rn(c, 0.375f))),
                              __fmul_rn(2.f, __fsqrt_rn(__fadd_rn(r, 0.375f))));
    return __fmul_rn(0.5f, __fmul_rn(d, d));
  }
}

// Moment-table index of a pooled count: nearest integer (ties to even),
// capped at MOMENT_NMAX.
__device__ __forceinline__ int count_index(float x) { return (int)rintf(fminf(x, (float)MOMENT_NMAX)); }

// Raw count [v / s_P]_+ of Eq. (raw-counts), as v times float(1 / s_P).
__device__ __forceinline__ float raw_count(float v, float inv) { return fmaxf(__fmul_rn(v, inv), 0.f); }

// x^kappa: the exponents of the paper's sensitivity grid (0.25, 0.5, 1, 2,
// 3, 4) by square roots and products, any other by powf.
__device__ __forceinline__ float pow_kappa(float x, float k) {
  if (k == 1.f) return x;
  if (k == 0.5f) return __fsqrt_rn(x);
  if (k == 0.25f) return __fsqrt_rn(__fsqrt_rn(x));
  if (k == 2.f) return __fmul_rn(x, x);
  if (k == 3.f) return __fmul_rn(__fmul_rn(x, x), x);
  if (k == 4.f) {
    const float x2 = __fmul_rn(x, x);
    return __fmul_rn(x2, x2);
  }
  return powf(x, k);
}

// Scores of the KB candidates q + b (b < KB, consecutive on the last axis)
// against the reference p, both in the staged guide with patch rows at
// rowoff: P d_m = sum_i phi_m(r_i, c_i) over the entries in C order, or,
// standardized, Z_m of Eq. (standardized-distance) with the moments at
// n_i = r_i + c_i (0 when their variances sum to 0).  The KB candidates are
// interleaved for instruction-level parallelism; each one's sum keeps the
// entry order.  Candidates past the window read the region's padding, as the
// SSD loop does; their scores are discarded (every table index stays in
// [0, MOMENT_NMAX] whatever they read).
template <int METRIC, bool STD, int KB>
__device__ __forceinline__ void metric_block(const DGeom &g, const float *p, const float *q, const int *rowoff,
                                             float (&acc)[KB]) {
  const float inv = g.inv_sp;
  float ms[KB], vs[KB];
#pragma unroll
  for (int b = 0; b < KB; ++b) { acc[b] = 0.f; ms[b] = 0.f; vs[b] = 0.f; }
  for (int r = 0; r < g.rows; ++r) {
    const float *pr = p + rowoff[r], *qr = q + rowoff[r];
    for (int i = 0; i < g.jL; ++i) {
      const float rv = raw_count(pr[i], inv);
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const float cv = raw_count(qr[i + b], inv);
        acc[b] = __fadd_rn(acc[b], poisson_phi<METRIC>(rv, cv));
        if (STD) {
          const float2 mv = __ldg(&g.mom[count_index(__fadd_rn(rv, cv))]);
          ms[b] = __fadd_rn(ms[b], mv.x);
          vs[b] = __fadd_rn(vs[b], mv.y);
        }
      }
    }
  }
  if (STD) {
#pragma unroll
    for (int b = 0; b < KB; ++b)
      acc[b] = vs[b] > 0.f ? __fdiv_rn(__fsub_rn(acc[b], ms[b]), __fsqrt_rn(vs[b])) : 0.f;
  }
}

template <int KB>
__device__ __forceinline__ void metric_scores(const DGeom &g, const float *p, const float *q, const int *rowoff,
                                              float (&acc)[KB]) {
  const bool st = g.policy == 2;
  switch (g.metric) {
    case 1:
      if (st) metric_block<1, true, KB>(g, p, q, rowoff, acc); else metric_block<1, false, KB>(g, p, q, rowoff, acc);
      break;
    case 2:
      if (st) metric_block<2, true, KB>(g, p, q, rowoff, acc); else metric_block<2, false, KB>(g, p, q, rowoff, acc);
      break;
    default:
      if (st) metric_block<3, true, KB>(g, p, q, rowoff, acc); else metric_block<3, false, KB>(g, p, q, rowoff, acc);
      break;
  }
}

// Reference finite-count threshold in sum units, P T_ref(p; t) of Eq.
// (reference-threshold): sum_i mu_m(2 r_i) + t sqrt(sum_i v_m(2 r_i)) +
// beta_s P r-bar^kappa_s, from the reference patch alone.
__device__ __noinline__ float metric_threshold(const DGeom &g, const float *p, const int *rowoff) {
  const float inv = g.inv_sp;
  float ms = 0.f, vs = 0.f, rs = 0.f;
  for (int r = 0; r < g.rows; ++r) {
    const float *pr = p + rowoff[r];
    for (int i = 0; i < g.jL; ++i) {
      const float rv = raw_count(pr[i], inv);
      const float2 mv = __ldg(&g.mom[count_index(__fmul_rn(2.f, rv))]);
      ms = __fadd_rn(ms, mv.x);
      vs = __fadd_rn(vs, mv.y);
      rs = __fadd_rn(rs, rv);
    }
  }
  const float rbar = __fdiv_rn(rs, (float)g.P);
  const float allow = __fmul_rn(g.beta_p, pow_kappa(rbar, g.kappa));
  return __fadd_rn(__fadd_rn(ms, __fmul_rn(g.mt, __fsqrt_rn(vs))), allow);
}

// Poisson distances on count data in exact integer arithmetic.  When every
// staged value of a tile is s_P times an integer count K <= PFIX_K / 2 (to
// within float rounding; Eq. raw-counts), the per-entry contributions come
// from fixed-point tables (units 2^-32) and a candidate's sums are exact
// 64-bit integers: they depend only on the multiset of its terms, and two
// candidates compare as the sums of their contributions rounded to the
// tables' 2^-33 compare.

// The count K of a staged value v (v * float(1 / s_P) rounded).
__device__ __forceinline__ int count_of(float v, float inv) { return max(__float2int_rn(v * inv), 0); }

// phi_m(r, c) of Eq. (varphi) at integer counts, units 2^-32:
// deviance 2 (r ln 2r + c ln 2c - n ln n), Pearson (r - c)^2 / n,
// Anscombe (A(c) - A(r))^2 / 2 with A(K) = 2 sqrt(K + 3/8).
template <int METRIC>
__device__ __forceinline__ long long phi_fix(const long long *__restrict__ T, int r, int c) {
  const int n = r + c;
  if (METRIC == 1) return 2 * (__ldg(T + PFIX_A + r) + __ldg(T + PFIX_A + c) - __ldg(T + PFIX_B + n));
  if (METRIC == 2) {
    if (n == 0) return 0;
    const unsigned long long d = (unsigned long long)abs(r - c);
    return (long long)__umul64hi((d * d) << 32, (unsigned long long)__ldg(T + PFIX_A + n));
  }
  const long long dA = __ldg(T + PFIX_A + c) - __ldg(T + PFIX_A + r);  // units 2^-44
  const unsigned long long ad = (unsigned long long)(dA < 0 ? -dA : dA);
  const unsigned long long lo = ad * ad, hi = __umul64hi(ad, ad);    // (dA)^2, units 2^-88
  return (long long)((hi << 7) | (lo >> 57));                         // / 2, units 2^-32
}

// Exact sums of the KB candidates q + b (b < KB) against the reference p:
// acc = sum phi, and for the standardized policy ms / vs = sum of the
// moments at the pooled counts (units 2^-32).
template <int METRIC, bool STD, int KB>
__device__ __forceinline__ void metric_block_fix(const DGeom &g, const float *p, const float *q, const int *rowoff,
                                                 long long (&acc)[KB], long long (&ms)[KB], long long (&vs)[KB]) {
  const float inv = g.inv_sp;
  const long long *T = g.pfix;
#pragma unroll
  for (int b = 0; b < KB; ++b) { acc[b] = 0; ms[b] = 0; vs[b] = 0; }
  for (int r = 0; r < g.rows; ++r) {
    const float *pr = p + rowoff[r], *qr = q + rowoff[r];
    for (int i = 0; i < g.jL; ++i) {
      const int rv = count_of(pr[i], inv);
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const int cv = count_of(qr[i + b], inv);
        acc[b] += phi_fix<METRIC>(T, rv, cv);
        if (STD) {
          const int n = min(rv + cv, MOMENT_NMAX);
          ms[b] += __ldg(T + PFIX_MU + n);
          vs[b] += __ldg(T + PFIX_V + n);
        }
      }
    }
  }
}

// The score of candidates from their exact sums: P d_m (fixed and reference
// policies) or Z_m of Eq. (standardized-distance), in float for the list
// (key) or in double for a decision.
__device__ __forceinline__ float pm_key(int policy, long long acc, long long ms, long long vs) {
  if (policy != 2) return __ll2float_rn(acc) * 2.3283064365386963e-10f;
  if (vs <= 0) return 0.f;
  return __ll2float_rn(acc - ms) * 1.52587890625e-05f * rsqrtf(__ll2float_rn(vs));
}
__device__ __forceinline__ double pm_score64(int policy, long long acc, long long ms, long long vs) {
  if (policy != 2) return ldexp(__ll2double_rn(acc), -32);
  if (vs <= 0) return 0.0;
  return ldexp(__ll2double_rn(acc - ms), -16) / sqrt(__ll2double_rn(vs));
}

template <int KB>
__device__ __forceinline__ void metric_keys_fix(const DGeom &g, const float *p, const float *q, const int *rowoff,
                                                float (&key)[KB]) {
  long long acc[KB], ms[KB], vs[KB];
  const bool st = g.policy == 2;
  switch (g.metric) {
    case 1:
      if (st) metric_block_fix<1, true, KB>(g, p, q, rowoff, acc, ms, vs);
      else metric_block_fix<1, false, KB>(g, p, q, rowoff, acc, ms, vs);
      break;
    case 2:
      if (st) metric_block_fix<2, true, KB>(g, p, q, rowoff, acc, ms, vs);
      else metric_block_fix<2, false, KB>(g, p, q, rowoff, acc, ms, vs);
      break;
    default:
      if (st) metric_block_fix<3, true, KB>(g, p, q, rowoff, acc, ms, vs);
      else metric_block_fix<3, false, KB>(g, p, q, rowoff, acc, ms, vs);
      break;
  }
#pragma unroll
  for (int b = 0; b < KB; ++b) key[b] = pm_key(g.policy, acc[b], ms[b], vs[b]);
}

// Double-precision score of one candidate (count data).
__device__ __noinline__ double pm_exact64(const DGeom &g, const float *p, const float *q, const int *rowoff) {
  long long acc[1], ms[1], vs[1];
  const bool st = g.policy == 2;
  switch (g.metric) {
    case 1:
      if (st) metric_block_fix<1, true, 1>(g, p, q, rowoff, acc, ms, vs);
      else metric_block_fix<1, false, 1>(g, p, q, rowoff, acc, ms, vs);
      break;
    case 2:
      if (st) metric_block_fix<2, true, 1>(g, p, q, rowoff, acc, ms, vs);
      else metric_block_fix<2, false, 1>(g, p, q, rowoff, acc, ms, vs);
      break;
    default:
      if (st) metric_block_fix<3, true, 1>(g, p, q, rowoff, acc, ms, vs);
      else metric_block_fix<3, false, 1>(g, p, q, rowoff, acc, ms, vs);
      break;
  }
  return pm_score64(g.policy, acc[0], ms[0], vs[0]);
}

// Reference finite-count threshold of Eq. (reference-threshold) in sum
// units, P T_ref = sum mu(2 r_i) + t sqrt(sum v(2 r_i)) + beta_s P r-bar^kappa,
// from exact sums over the reference patch; in float (t32) and double (t64).
__device__ __noinline__ void pm_threshold(const DGeom &g, const float *p, const int *rowoff, float *t32,
                                          double *t64) {
  const float inv = g.inv_sp;
  const long long *T = g.pfix;
  long long ms = 0, vs = 0, rs = 0;
  for (int r = 0; r < g.rows; ++r) {
    const float *pr = p + rowoff[r];
    for (int i = 0; i < g.jL; ++i) {
      const int rv = count_of(pr[i], inv);
      const int n = min(2 * rv, MOMENT_NMAX);
      ms += __ldg(T + PFIX_MU + n);
      vs += __ldg(T + PFIX_V + n);
      rs += rv;
    }
  }
  if (t32) {
    const float rbar = (float)rs / (float)g.P;
    *t32 = __ll2float_rn(ms) * 2.3283064365386963e-10f +
           g.mt * sqrtf(__ll2float_rn(vs) * 2.3283064365386963e-10f) + g.beta_p * pow_kappa(rbar, g.kappa);
  }
  if (t64) {
    const double rbar = (double)rs / (double)g.P;
    *t64 = ldexp(__ll2double_rn(ms), -32) + (double)g.mt64 * sqrt(ldexp(__ll2double_rn(vs), -32)) +
           g.beta_p64 * pow(rbar, g.kappa64);
  }
}

// ---------------------------------------------------------------------------
// block matching of one reference (Sec. 4.2 / 4.4, App. A group rules)
// ---------------------------------------------------------------------------

// Double-precision score of one candidate: Eq. (ssd) minus gamma times the
// noise bias (Def. "Noise-bias-corrected SSD"), evaluated as the definition
// reads: patch entries in C order, every difference, square, sum and
// product rounded once in double precision (no fused operations).  rb / cb:
// region offsets of the reference and the candidate patch.
__device__ __forceinline__ double ssd_score64(const DGeom &g, const float *__restrict__ S, const int *rowoff,
                                              int rb, int cb) {
  double ssd = 0.0, bias = 0.0;
  const bool pb = g.poisson && g.gamma64 != 0.0;
  for (int r = 0; r < g.rows; ++r) {
    const float *pr = S + rb + rowoff[r], *qr = S + cb + rowoff[r];
    for (int i = 0; i < g.jL; ++i) {
      const double p = pr[i], q = qr[i];
      const double d = __dsub_rn(q, p);
      ssd = __dadd_rn(ssd, __dmul_rn(d, d));
      if (pb) {
        const double t = __dadd_rn(p, q);
        bias = __dadd_rn(bias, t > 0.0 ? t : 0.0);
      }
    }
  }
  const double B = pb ? __dmul_rn(g.s_p64, bias) : g.gbias64;
  return __dsub_rn(ssd, __dmul_rn(g.gamma64, B));
}

// Exact integer arithmetic on a tile's guide values.  Every staged value is
// an integer multiple of q0 = 2^emin (emin: the lowest set-bit exponent over
// the tile) of magnitude below 2^span q0.  fixed_of returns v / q0.
__device__ __forceinline__ long long fixed_of(float v, int emin) {
  const unsigned b = __float_as_uint(v);
  const int ex = (int)((b >> 23) & 0xffu);
  const long long m = (long long)((b & 0x7fffffu) | (ex ? 0x800000u : 0u));
  const int sh = (ex ? ex : 1) - 150 - emin;  // v = m 2^(ex - 150)
  const long long r = sh >= 0 ? (m << sh) : (m >> -sh);
  return (b >> 31) ? -r : r;
}

// The unsigned 128-bit integer hi 2^64 + lo rounded once to double (the top
// 64 bits, with a sticky bit for the rest, converted with round-to-nearest-
// even: the sticky bit lies far below the rounding position).
__device__ __forceinline__ double u128_to_double(unsigned long long hi, unsigned long long lo) {
  if (hi == 0ull) return __ull2double_rn(lo);
  const int lz = __clzll((long long)hi);
  const unsigned long long top = lz ? ((hi << lz) | (lo >> (64 - lz))) : hi;
  const unsigned long long rest = lo << lz;
  return ldexp(__ull2double_rn(top | (rest != 0ull ? 1ull : 0ull)), 64 - lz);
}

// Double-precision score of one candidate from exact sums (the terms of
// Eq. ssd and of the Poisson bias summed exactly, then rounded once, as the
// oracle does): the SSD in units of q0^2 as a 128-bit integer, the bias sum
// in units of q0, then B = s_P bias and score = ssd - gamma B (Def.
// "Noise-bias-corrected SSD").  span <= 31: the differences fit 32 bits and
// their squares 64; span <= 51: 64-bit differences, 128-bit squares, and the
// bias sum of P <= 1024 entries stays below 2^63.  The sums depend only on
// the multiset of the terms.
__device__ __forceinline__ double ssd_score_exact(const DGeom &g, const float *__restrict__ S, const int *rowoff,
                                                  int rb, int cb, int emin, int span) {
  unsigned long long lo = 0ull, hi = 0ull;
  long long bsum = 0;
  const bool pb = g.poisson && g.gamma64 != 0.0;
  if (span <= 30 && emin >= -126) {
    // 32-bit path: v / q0 is an integer below 2^30 (a float scaled by a
    // power of two that is itself a normal float, so the conversion is
    // exact), differences and sums fit 32 bits, squares 64
    const float sc = ldexpf(1.f, -emin);
    for (int r = 0; r < g.rows; ++r) {
      const float *pr = S + rb + rowoff[r], *qr = S + cb + rowoff[r];
#pragma unroll 4
      for (int i = 0; i < g.jL; ++i) {
        const int ip = __float2int_rn(pr[i] * sc), iq = __float2int_rn(qr[i] * sc);
        const unsigned ud = (unsigned)abs(iq - ip);
        const unsigned long long sq = (unsigned long long)ud * ud;
        lo += sq;
        hi += lo < sq ? 1ull : 0ull;
        if (pb) bsum += max(ip + iq, 0);
      }
    }
    const double ssd = ldexp(u128_to_double(hi, lo), 2 * emin);
    const double B = pb ? __dmul_rn(g.s_p64, ldexp(__ll2double_rn(bsum), emin)) : g.gbias64;
    return __dsub_rn(ssd, __dmul_rn(g.gamma64, B));
  }
  const bool narrow = span <= 31;
  for (int r = 0; r < g.rows; ++r) {
    const float *pr = S + rb + rowoff[r], *qr = S + cb + rowoff[r];
    for (int i = 0; i < g.jL; ++i) {
      const long long ip = fixed_of(pr[i], emin), iq = fixed_of(qr[i], emin);
      const long long d = iq - ip;
      const unsigned long long ud = (unsigned long long)(d < 0 ? -d : d);
      unsigned long long sq_lo, sq_hi;
      if (narrow) {
        sq_lo = ud * ud;
        sq_hi = 0ull;
      } else {
        sq_lo = ud * ud;
        sq_hi = __umul64hi(ud, ud);
      }
      lo += sq_lo;
      hi += sq_hi + (lo < sq_lo ? 1ull : 0ull);
      if (pb) {
        const long long t = ip + iq;
        bsum += t > 0 ? t : 0;
      }
    }
  }
  const double ssd = ldexp(u128_to_double(hi, lo), 2 * emin);
  const double B = pb ? __dmul_rn(g.s_p64, ldexp(__ll2double_rn(bsum), emin)) : g.gbias64;
  return __dsub_rn(ssd, __dmul_rn(g.gamma64, B));
}

__device__ __noinline__ double ssd_score64_call(const DGeom &g, const float *__restrict__ S, const int *rowoff, int rb,
                                                int cb) {
  return ssd_score64(g, S, rowoff, rb, cb);
}

// Score of a candidate for a double-precision decision: exact sums where the
// tile's span allows (span <= 51), else the sequential double sum.
__device__ __forceinline__ double score_decide(const DGeom &g, const float *__restrict__ S, const int *rowoff, int rb,
                                               int cb, int emin, int span) {
  return span <= 51 ? ssd_score_exact(g, S, rowoff, rb, cb, emin, span) : ssd_score64_call(g, S, rowoff, rb, cb);
}

// Double-precision score of a candidate for a decision: SSD (score_decide)
// or, on count data, a Poisson distance (pm_exact64).
__device__ __forceinline__ double cand_score64(const DGeom &g, const float *__restrict__ S, const int *rowoff, int rb,
                                               int cb, int emin, int span, bool pm) {
  return pm ? pm_exact64(g, S + rb, S + cb, rowoff) : score_decide(g, S, rowoff, rb, cb, emin, span);
}

// Every candidate of a window (window indices 0..ncand-1, region offsets
// from the window origin lo and extents W) scored in double precision;
// returns this lane's entry of the sorted list of the 32 best by (score,
// window index), the reference (ridx) left out.
template <int D>
__device__ __noinline__ void full_window(const DGeom &g, const float *__restrict__ S, const int *rowoff, int lane,
                                         int rbase, int ridx, int ncand, const int *lo, const int *W, int emin,
                                         int span, bool pm, double &fk, int &fi) {
  fk = DBL_MAX;
  fi = INT_MAX;
  for (int c0 = 0; c0 < ncand; c0 += 32) {
    const int c = c0 + lane;
    double sc = DBL_MAX;
    int wi = INT_MAX;
    if (c < ncand && c != ridx) {
      int rem = c, off = 0;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) {
        const int x = rem % W[d];
        rem /= W[d];
        off += (lo[d] + x) * g.rst[d];
      }
      sc = cand_score64(g, S, rowoff, rbase, off, emin, span, pm);
      wi = c;
    }
    warp_sort(sc, wi, lane);
    warp_merge(fk, fi, sc, wi, lane);
  }
}

// The group of one reference from the warp's FP32 list (lk, li): the best
// candidates by (FP32 score, window index), one per lane, sorted; past the
// valid entries (li = INT_MAX) the list is empty.  Ranking and acceptance
// (App. A group rules) are decided as the double-precision definition
// decides them.  Every FP32 score s carries an error bound ku (|s| + 2 gamma
// Bm) (Bm: a bound on the noise bias of every candidate), so each list
// entry is an interval; the entries split into runs between the gaps where
// every interval to the left lies below every interval to the right (prefix
// maximum of the upper ends against the suffix minimum of the lower ends).
// A run of two or more entries that reaches a group position (the first
// M - 1), and a group position whose interval holds tau, are rescored in
// double precision (decide_refine); candidates outside the list (never
// offered: FP32 score above the final offer threshold thr; or pushed out:
// at least the last entry) are bounded below, and if that bound reaches the
// upper ends of the group positions, the whole window is scored in double
// precision.  exact: the tile's data are dyadic and every FP32 score is
// exact.  Returns the number of accepted list entries among the first
// M - 1 (the accepted candidates are a prefix of the sorted list); li may be
// reordered.

// The rare part: rescoring of the flagged entries (resc) or of the whole
// window (full), the list sorted again in double precision, and the
// acceptance count.
template <int D>
__device__ __noinline__ int decide_refine(const DGeom &g, const float *__restrict__ S, const int *rr,
                                          const int *org, const int *rowoff, int lane, int rbase, int ridx,
                                          int ncand, int nl, int KK, bool resc, bool full, int emin, int span,
                                          bool pm, float lk, int &li) {
  const unsigned FULL = 0xffffffffu;
  int lo[D], W[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int rglob = rr[d] + org[d];
    const int l = max(rglob - g.rad[d], 0);
    const int h = (int)min((int64_t)rglob + g.rad[d], g.ell[d]);
    lo[d] = l - org[d];
    W[d] = h - l + 1;
  }
  double key = lane < nl ? (double)lk : DBL_MAX;
  if (full) {
    full_window<D>(g, S, rowoff, lane, rbase, ridx, ncand, lo, W, emin, span, pm, key, li);
    if (g.diag && lane == 0) atomicAdd(g.diag + 1, 1ull);
  } else {
    int off = 0;
    {
      int rem = li;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) {
        const int c = rem % W[d];
        rem /= W[d];
        off += (lo[d] + c) * g.rst[d];
      }
    }
    if (resc) key = cand_score64(g, S, rowoff, rbase, off, emin, span, pm);
    if (g.diag) {
      const int nr = __popc(__ballot_sync(FULL, resc));
      if (lane == 0) atomicAdd(g.diag, (unsigned long long)nr);
    }
    warp_sort(key, li, lane);
  }
  // acceptance: score < tau (App. A; Sec. 4.3 for the Poisson distances),
  // in double precision
  double t64 = g.tau64;
  if (pm && g.policy == 1) pm_threshold(g, S + rbase, rowoff, nullptr, &t64);
  return __popc(__ballot_sync(FULL, lane < KK && key < t64));
}

template <int D>
__device__ __forceinline__ int decide_group(const DGeom &g, const float *__restrict__ S, const int *rr, const int *org,
                                            const int *rowoff, int lane, int rbase, int ridx, int ncand, float Bm,
                                            float thr, bool exact, int emin, int span, bool pm, float tau32,
                                            float tbr, float lk, int &li) {
  const unsigned FULL = 0xffffffffu;
  const int K = g.M - 1;
  const int navail = ncand - 1;
  const int nl = __popc(__ballot_sync(FULL, li != INT_MAX));  // valid list entries (a prefix)
  const int KK = min(K, nl);
  // tau bracketed in float: below tlo certainly accepted, at or above thi
  // certainly not
  const float tlo = tau32 - fabsf(tau32) * tbr, thi = tau32 + fabsf(tau32) * tbr;
  if (exact || KK <= 0) {
    // exact FP32 scores: only a score within a float step of tau needs the
    // double-precision comparison
    const bool amb = lane < KK && lk >= tlo && lk < thi;
    const bool acc = lane < KK && (lk < tlo || (amb && (double)lk < g.tau64));
    return __popc(__ballot_sync(FULL, acc));
  }
  const float gam = g.gamma;
  // |s32 - s| <= ku (ssd + gamma B) <= ku (|s32| + 2 gamma Bm)
  const float dl = lane < nl ? g.ku * (fabsf(lk) + 2.f * gam * Bm) : 0.f;
  const float flo = lane < nl ? lk - dl : FLT_MAX;
  const float fhi = lane < nl ? lk + dl : -FLT_MAX;
  const float lk31 = __shfl_sync(FULL, lk, 31);
  const float kout = nl == 32 ? fminf(thr, lk31) : thr;
  const float outlb = navail > nl ? kout - g.ku * (fabsf(kout) + 2.f * gam * Bm) : FLT_MAX;
  float pmax = fhi, smin = flo;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float a = __shfl_up_sync(FULL, pmax, o);
    const float b = __shfl_down_sync(FULL, smin, o);
    if (lane >= o) pmax = fmaxf(pmax, a);
    if (lane + o < 32) smin = fminf(smin, b);
  }
  const float snext = __shfl_down_sync(FULL, smin, 1);
  // gap after position `lane` open (every interval to its left below every
  // list interval to its right); positions past the list are empty
  const unsigned G = __ballot_sync(FULL, lane + 1 >= nl || pmax < snext);
  const unsigned below = G & ((1u << lane) - 1u);
  const int a = below ? 32 - __clz(below) : 0;             // first position of this run
  const unsigned atabove = G & (~0u << lane);
  const int b = atabove ? __ffs(atabove) - 1 : 32;         // last position of this run
  const bool relevant = lane < nl && a <= KK - 1;
  const bool tamb = lane < KK && flo < thi && fhi >= tlo;
  const bool resc = (relevant && b > a) || tamb;
  // the (M-1)-th smallest exact score is at most the largest upper end among
  // the first M - 1 entries; a candidate outside the list whose lower bound
  // stays above it cannot enter the group
  const float hull = __shfl_sync(FULL, pmax, KK - 1);
  const bool full = outlb <= hull;
  if (full || __any_sync(FULL, resc))
    return decide_refine<D>(g, S, rr, org, rowoff, lane, rbase, ridx, ncand, nl, KK, resc, full, emin, span, pm, lk,
                            li);
  return __popc(__ballot_sync(FULL, lane < KK && lk < tlo));
}

// Squared distances and noise-bias sums of the KB candidates q + b (b < KB,
// consecutive on the last axis) against the reference p, over all patch
// rows of JJ entries (Sec. 4.1: the SSD and the B term of the stage-1
// distance).  bs sums [p + q]_+, or p + q when every value is >= 0
// (NONNEG).
template <int KB, int JJ, bool NONNEG>
__device__ __forceinline__ void ssd_bias_rows(const float *__restrict__ p, const float *__restrict__ q,
                                              const int *__restrict__ rowoff, int rows, float *acc, float *bs) {
  constexpr int IB = JJ < 8 ? JJ : 8;
  float a[KB], t[KB];
#pragma unroll
  for (int b = 0; b < KB; ++b) { a[b] = 0.f; t[b] = 0.f; }
  for (int r = 0; r < rows; ++r) {
    const float *prow = p + rowoff[r];
    const float *qrow = q + rowoff[r];
    float w[KB];
#pragma unroll
    for (int b = 0; b < KB - 1; ++b) w[b] = qrow[b];
#pragma unroll 1
    for (int i0 = 0; i0 < JJ; i0 += IB) {
#pragma unroll
      for (int ii = 0; ii < IB; ++ii) {
        const int i = i0 + ii;
        w[KB - 1] = qrow[i + KB - 1];
        const float pv = prow[i];
#pragma unroll
        for (int b = 0; b < KB; ++b) {
          const float df = __fsub_rn(w[b], pv);
          a[b] = fmaf(df, df, a[b]);
          const float sp = __fadd_rn(pv, w[b]);
          t[b] = __fadd_rn(t[b], NONNEG ? sp : fmaxf(sp, 0.f));
        }
#pragma unroll
        for (int b = 0; b < KB - 1; ++b) w[b] = w[b + 1];
      }
    }
  }
#pragma unroll
  for (int b = 0; b < KB; ++b) { acc[b] = a[b]; bs[b] = t[b]; }
}

// The same out of line, for the planar kernels: only their tiles without
// the patch-sum map take it, and inlined beside the plain SSD loop it costs
// the stage kernel registers.  The 3-D kernels (no patch-sum map) inline it.
template <int KB, int JJ>
__device__ __noinline__ void ssd_bias_block(const float *__restrict__ p, const float *__restrict__ q,
                                            const int *__restrict__ rowoff, int rows, bool nonneg, float *acc,
                                            float *bs) {
  if (nonneg) ssd_bias_rows<KB, JJ, true>(p, q, rowoff, rows, acc, bs);
  else ssd_bias_rows<KB, JJ, false>(p, q, rowoff, rows, acc, bs);
}

template <int D, int JL, int KB, int ST>
// nonneg: every staged guide value is >= 0 (count data), where
// [p + q]_+ = p + q exactly and the bias term skips the max.
// exact: every staged guide value lies on a dyadic grid fine enough that
// the FP32 scores are exact (decide_group).
__device__ __forceinline__ int warp_match(const DGeom &g, const float *__restrict__ S, const int *rr,
                          const int *org, const int *rowoff, int lane, int *mem, bool nonneg, bool exact,
                          int emin, int span, float vmaxf, bool counts, unsigned long long *diag,
                          const float *__restrict__ bsm) {
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
  const float gam = g.gamma;
  // Poisson matching distances in stage 1 (Secs. 4.2-4.3): the generic
  // kernels, or the cubic-patch kernels instantiated with ST = 3
  const bool pmetric = (JL == 0 || ST == 3) && ST != 2 && g.metric != 0;
  // count data: exact integer sums (metric_keys_fix) and double-precision
  // decisions; otherwise the FP32 scores decide
  const bool pfix = pmetric && counts && g.pfix != nullptr;
  float tau = g.tau;
  if (pmetric && g.policy == 1) {
    if (pfix) pm_threshold(g, S + rbase, rowoff, &tau, nullptr);
    else tau = metric_threshold(g, S + rbase, rowoff);
  }
  const float gbias = g.poisson ? 0.f : __fmul_rn(__fmul_rn(2.f, (float)g.P), g.var_g);
  float lk = FLT_MAX;
  int li = INT_MAX;
  float thr = FLT_MAX;
  int thri = INT_MAX;
  int nacc = 0;
  // Offers must beat the (M-1)-th list entry widened by the error bounds of
  // the FP32 scores (decide_group): lk[M-2] + 3 ku (|lk[M-2]| + 2 gamma Bm),
  // Bm a bound on the noise bias of every candidate (Poisson: s_P times the
  // reference's sum plus P times the tile's largest value; Gaussian: 2 P
  // sigma^2).  The widened threshold only falls as the list improves, and a
  // candidate that was never offered has a lower bound above the upper ends
  // of the first M - 1 entries, so it cannot belong to the group in double
  // precision.  Exact tiles take no margin.
  const int KP = g.M >= 2 ? g.M - 2 : 0;
  float Bm = 0.f;
  if (!pmetric && gam > 0.f) {
    if (g.poisson) {
      float ps = 0.f;
      for (int e = lane; e < g.P; e += 32) ps += fmaxf(S[rbase + rowoff[e / g.jL] + e % g.jL], 0.f);
      Bm = g.s_p * (warp_sum(ps) + (float)g.P * vmaxf);
    } else {
      Bm = 2.f * (float)g.P * g.var_g;
    }
  }
  const float kmar = (exact || (pmetric && !pfix)) ? 0.f : 3.f * g.ku;
  int iters = (total + 31) / 32;
  // the iterations from the one holding the reference outwards, alternating
  // after and before it: near candidates tend to score low, so the offer
  // threshold falls early (the list is the same in any order)
  int itc;
  {
    const int oref = ridx / WL;
    itc = min((oref * nchk + (ridx - oref * WL) / KB) / 32, iters - 1);
  }
  for (int s = 0, nlo = itc - 1, nhi = itc + 1; s < iters; ++s) {
    int it = itc;
    if (s > 0) {
      bool up = (s & 1) != 0;
      if (up && nhi >= iters) up = false;
      if (!up && nlo < 0) up = true;
      it = up ? nhi++ : nlo--;
    }
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
      if (pfix) metric_keys_fix<KB>(g, S + rbase, S + cbase, rowoff, acc);
      else if (pmetric) metric_scores<KB>(g, S + rbase, S + cbase, rowoff, acc);
      if (JL > 0 && ST != 2 && !pmetric && g.bias_on && bsm == nullptr) {
        if (D == 3) {
          if (nonneg) ssd_bias_rows<KB, JL, true>(S + rbase, S + cbase, rowoff, g.rows, acc, bs);
          else ssd_bias_rows<KB, JL, false>(S + rbase, S + cbase, rowoff, g.rows, acc, bs);
        } else {
          float ta[KB], tb[KB];
          ssd_bias_block<KB, JL>(S + rbase, S + cbase, rowoff, g.rows, nonneg, ta, tb);
#pragma unroll
          for (int b = 0; b < KB; ++b) { acc[b] = ta[b]; bs[b] = tb[b]; }
        }
      }
      const int rows_plain = pmetric || (JL > 0 && ST != 2 && g.bias_on && bsm == nullptr) ? 0 : g.rows;
      for (int r = 0; r < rows_plain; ++r) {
        const float *prow = S + rbase + rowoff[r];
        const float *qrow = S + cbase + rowoff[r];
        if (JL > 0) {
          // sliding window over the candidate row, q[b] = qrow[i + b],
          // unrolled in blocks of IB entries
          constexpr int JJ = JL > 0 ? JL : 1;
          constexpr int IB = JJ < 8 ? JJ : 8;
          float q[KB];
#pragma unroll
          for (int b = 0; b < KB - 1; ++b) q[b] = qrow[b];
#pragma unroll 1
          for (int i0 = 0; i0 < JJ; i0 += IB) {
#pragma unroll
            for (int ii = 0; ii < IB; ++ii) {
              const int i = i0 + ii;
              q[KB - 1] = qrow[i + KB - 1];
              const float pv = prow[i];
#pragma unroll
              for (int b = 0; b < KB; ++b) {
                float df = __fsub_rn(q[b], pv);
                acc[b] = fmaf(df, df, acc[b]);
              }
#pragma unroll
              for (int b = 0; b < KB - 1; ++b) q[b] = q[b + 1];
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
              if (ST != 2 && g.bias_on) bs[b] = __fadd_rn(bs[b], fmaxf(__fadd_rn(pv, qv), 0.f));
            }
          }
        }
      }
      if (JL > 0 && bsm != nullptr) {
        // the bias sums from the patch-sum map (sum p + sum q, all terms >= 0)
        const float ps = bsm[rbase];
#pragma unroll
        for (int b = 0; b < KB; ++b) bs[b] = b < kb ? ps + bsm[cbase + b] : 0.f;
      }
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        bool ok = b < kb && (widx0 + b) != ridx;
        // rounded exactly as written: no contraction of gam * B into the subtraction
        float B = g.poisson ? __fmul_rn(g.s_p, bs[b]) : gbias;
        float sc = gam > 0.f && !pmetric ? __fsub_rn(acc[b], __fmul_rn(gam, B)) : acc[b];
        if (ok) {
          key[b] = sc;
          idx[b] = widx0 + b;
          nacc += sc < tau;
        }
      }
    }
    // offer the candidates below the threshold, every lane its smallest
    // pending one per round; a lane whose smallest no longer beats the
    // threshold (which only falls) drops the rest.  The running list keeps
    // its 32 smallest (score, index) entries whatever the order of the
    // offers, so it ends as the 32 smallest candidates of the window.
    unsigned pend = 0u;
#pragma unroll
    for (int b = 0; b < KB; ++b)
      if (kv_less(key[b], idx[b], thr, thri)) pend |= 1u << b;
#pragma unroll 1
    while (__any_sync(0xffffffffu, pend != 0u)) {
      // the lane's smallest pending (score, index): a tree over its slots
      float ek[KB];
      int ei[KB], eb[KB];
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const bool pb = (pend >> b) & 1u;
        ek[b] = pb ? key[b] : FLT_MAX;
        ei[b] = pb ? idx[b] : INT_MAX;
        eb[b] = b;
      }
#pragma unroll
      for (int w = 1; w < KB; w *= 2) {
#pragma unroll
        for (int b = 0; b + w < KB; b += 2 * w) {
          if (kv_less(ek[b + w], ei[b + w], ek[b], ei[b])) {
            ek[b] = ek[b + w];
            ei[b] = ei[b + w];
            eb[b] = eb[b + w];
          }
        }
      }
      const float ck = ek[0];
      const int ci = ei[0];
      const bool has = ci != INT_MAX;
      const bool offer = has && kv_less(ck, ci, thr, thri);
      if (has) pend = offer ? (pend & ~(1u << eb[0])) : 0u;
      unsigned omask = __ballot_sync(0xffffffffu, offer);
      if (omask) {
        if (__popc(omask) <= 8) {
          // few offers: insert them one at a time (the list keeps its 32
          // smallest entries, as the merge does)
          while (omask) {
            const int src = __ffs(omask) - 1;
            omask &= omask - 1;
            const float sk = __shfl_sync(0xffffffffu, ck, src);
            const int si = __shfl_sync(0xffffffffu, ci, src);
            const int pos = __popc(__ballot_sync(0xffffffffu, kv_less(lk, li, sk, si)));
            const float uk = __shfl_up_sync(0xffffffffu, lk, 1);
            const int ui = __shfl_up_sync(0xffffffffu, li, 1);
            if (lane > pos) { lk = uk; li = ui; }
            else if (lane == pos) { lk = sk; li = si; }
          }
        } else {
          float ok = offer ? ck : FLT_MAX;
          int oi = offer ? ci : INT_MAX;
          warp_sort(ok, oi, lane);
          warp_merge(lk, li, ok, oi, lane);
        }
        {
          const float t = __shfl_sync(0xffffffffu, lk, KP);
          thri = __shfl_sync(0xffffffffu, li, KP);
          if (kmar > 0.f && t != FLT_MAX) {
            thr = t + kmar * (fabsf(t) + 2.f * gam * Bm);
            thri = INT_MAX;
          } else {
            thr = t;
          }
        }
      }
    }
  }
  int K = g.M - 1;
  int navail = (int)ncand - 1;
  int take;
  if (pmetric && !pfix) {
    take = min(warp_sum_i(nacc), K);
  } else {
    // tau bracket: the float tau of the host (relative 2^-22), or the FP32
    // reference threshold of pm_threshold (relative 2^-18)
    const float tbr = pfix && g.policy == 1 ? 3.8147e-6f : 2.4e-7f;
    take = decide_group<D>(g, S, rr, org, rowoff, lane, rbase, ridx, (int)ncand, Bm, thr, exact, emin, span, pfix,
                           tau, tbr, lk, li);
  }
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
// collaborative filtering of one group (Secs. 5-7)
// ---------------------------------------------------------------------------

// Diagonal factor of the windowed synthesis metric (Def. "Windowed synthesis
// metrics") for spatial coefficient v, C order over the patch axes: the
// separable product prod_d wsyn[d][q_d].
__device__ __forceinline__ float syn_energy(const DGeom &g, int v) {
  float e = 1.f;
  for (int d = g.D - 1; d >= 0; --d) {
    const int jd = g.j[d];
    const int q = v % jd;
    v /= jd;
    e *= g.wsyn[d][q];
  }
  return e;
}

// Entry (l, m) of the group-axis transform of n members: Haar rows ordered
// [scaling, coarsest detail, ..., finest details], or the DCT-II from the
// global table.
__device__ __forceinline__ float group_axis_entry(const DGeom &g, const float *tab, int n, int l, int m) {
  if (g.gtrans != 0) return __ldg(tab + gen_off(n) + l * n + m);
  if (l == 0) return rsqrtf((float)n);
  const int s = 31 - __clz(l);          // level: l in [2^s, 2^(s+1))
  const int b = n >> s, r = l - (1 << s);
  if (m < r * b || m >= (r + 1) * b) return 0.f;
  const float v = rsqrtf((float)b);
  return m < r * b + b / 2 ? v : -v;
}

// Def. "Partial shared-source Poisson variance model" for the leading kex
// group-axis planes, in per-location form.  The diagonal model sum_i T_ki^2
// m_v(u_i) (T_(l,q),(m,p) = A0[l][m] F_q(p)) counts every entry's own weight
// once; the exact variance sums over the distinct source locations u the
// squared effective weight t_ku = sum of the weights a_i of the entries taken
// from u (Def. "Effective transform weights").  The two differ only at
// locations covered by two or more members, so each such u adds
// m_v(u) (t_ku^2 - sum_i a_i^2).  One pass over the group: overlap masks of
// the members by ballot; per member m, its entries (lanes) covered by a
// later overlapping member and by no earlier one are the shared locations
// that m owns; each is then processed by the whole warp with lanes over the
// spatial coefficients q (NS per lane: q = 32 s0 + lane + 32 h, h < NS),
// reading the transposed analysis factors F^T (block 3 of the shared axis
// matrices).  With the Haar group transform the planes l0..l0+3 < 4 are
// signed sums of the four member quarters, so a covering entry costs one
// weight F_q and two accumulations; otherwise the group-axis entries of the
// four planes come from the member lanes.  corr[h][k] receives the
// correction of plane l0 + k (planes >= min(kex, n) stay 0).  vcrd:
// patch-entry coordinates, 5 bits per axis.  Returns the largest number of
// members covering one location (for the FP32 error band).
template <int D, int NS>
__device__ __noinline__ int shared_source_pass(const DGeom &g, int n, int lane, int s0, int l0,
                                               const int *__restrict__ mem, const int *__restrict__ vreg,
                                               const int *__restrict__ vcrd, const float *__restrict__ Sg,
                                               const float *mats, const int *moff, const float *tab,
                                               float (&corr)[NS][4]) {
  const unsigned FULL = 0xffffffffu;
  const int L = min(g.kex, n);
#pragma unroll
  for (int h = 0; h < NS; ++h)
#pragma unroll
    for (int k = 0; k < 4; ++k) corr[h][k] = 0.f;
  if (n < 2 || l0 >= L) return 1;
  int J[D];
  const float *FT[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    J[d] = g.j[d];
    FT[d] = mats + moff[d] + 3 * J[d] * J[d];
  }
  // lane m: region coordinates of member m and its overlap mask
  int cm[D];
#pragma unroll
  for (int d = 0; d < D; ++d) cm[d] = lane < n ? (mem[lane] / g.rst[d]) % g.RGP[d] : 0;
  unsigned ov = 0u;
  for (int m = 0; m < n; ++m) {
    // every lane takes part in every shuffle (none under a condition)
    bool o = lane < n && lane != m;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int c = __shfl_sync(FULL, cm[d], m);
      o = o && abs(cm[d] - c) < J[d];
    }
    const unsigned b = __ballot_sync(FULL, o);
    if (lane == m) ov = b;
  }
  if (__ballot_sync(FULL, ov != 0u) == 0u) return 1;
  const bool haar = g.gtrans == 0 && L <= 4;
  // member quarter of the Haar planes: m >> (log2 n - 2), n = 2: 2 m
  const int tn = 31 - __clz(n);
  const int qshl = tn >= 2 ? 0 : 2 - tn, qshr = tn >= 2 ? tn - 2 : 0;
  const float r1 = rsqrtf((float)n), r2 = sqrtf(2.f / (float)n);
  // group-axis entries of planes l0..l0+3 held by the member lanes
  float a0[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a0[k] = (!haar && lane < n && l0 + k < L) ? group_axis_entry(g, tab, n, l0 + k, lane) : 0.f;
  // this lane's coefficients and their axis coordinates
  int qc[NS][D];
#pragma unroll
  for (int h = 0; h < NS; ++h) {
    const int q = 32 * (s0 + h) + lane;
    const int c = q < g.P ? vcrd[q] : 0;
#pragma unroll
    for (int d = 0; d < D; ++d) qc[h][d] = (c >> (5 * d)) & 31;
  }
  int cmax = 1;
  for (int m = 0; m < n; ++m) {
    const unsigned ovm = __shfl_sync(FULL, ov, m);
    if (ovm == 0u) continue;
    int cmm[D];
#pragma unroll
    for (int d = 0; d < D; ++d) cmm[d] = __shfl_sync(FULL, cm[d], m);
    const unsigned earlier = (1u << m) - 1u;
    for (int p0 = 0; p0 < g.P; p0 += 32) {
      const int p = p0 + lane;
      const int pc = p < g.P ? vcrd[p] : 0;
      int ud[D];  // location coordinates of this lane's entry of m
#pragma unroll
      for (int d = 0; d < D; ++d) ud[d] = ((pc >> (5 * d)) & 31) + cmm[d];
      unsigned cover = 0u;
      for (unsigned r = ovm; r; r &= r - 1u) {
        const int m2 = __ffs(r) - 1;
        bool in = p < g.P;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int c2 = __shfl_sync(FULL, cm[d], m2);
          in = in && (unsigned)(ud[d] - c2) < (unsigned)J[d];
        }
        if (in) cover |= 1u << m2;
      }
      unsigned todo = __ballot_sync(FULL, cover != 0u && (cover & earlier) == 0u);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1u;
        const unsigned cv = __shfl_sync(FULL, cover, src) | (1u << m);
        int us[D];
#pragma unroll
        for (int d = 0; d < D; ++d) us[d] = __shfl_sync(FULL, ud[d], src);
        cmax = max(cmax, __popc(cv));
        const float mv = g.s_p * fmaxf(Sg[mem[m] + vreg[p0 + src]], 0.f);
        float Q[NS][4], R[NS][4];
#pragma unroll
        for (int h = 0; h < NS; ++h)
#pragma unroll
          for (int k = 0; k < 4; ++k) Q[h][k] = R[h][k] = 0.f;
        for (unsigned r = cv; r; r &= r - 1u) {
          const int m2 = __ffs(r) - 1;
          float f[NS];
#pragma unroll
          for (int h = 0; h < NS; ++h) f[h] = 1.f;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const float *row = FT[d] + (us[d] - __shfl_sync(FULL, cm[d], m2)) * J[d];
#pragma unroll
            for (int h = 0; h < NS; ++h) f[h] *= row[qc[h][d]];
          }
          if (haar) {
            switch ((m2 << qshl) >> qshr) {
#define BMND_Q(K)                                                       \
  case K:                                                               \
    _Pragma("unroll") for (int h = 0; h < NS; ++h) {                    \
      Q[h][K] += f[h];                                                  \
      R[h][K] = fmaf(f[h], f[h], R[h][K]);                              \
    }                                                                   \
    break;
              BMND_Q(0) BMND_Q(1) BMND_Q(2) BMND_Q(3)
#undef BMND_Q
            }
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float a = __shfl_sync(FULL, a0[k], m2);
#pragma unroll
              for (int h = 0; h < NS; ++h) {
                const float x = a * f[h];
                Q[h][k] += x;
                R[h][k] = fmaf(x, x, R[h][k]);
              }
            }
          }
        }
#pragma unroll
        for (int h = 0; h < NS; ++h) {
          float t[4], sq[4];
          if (haar) {
            // planes 0..3 of the Haar rows: all members, the two halves,
            // the quarters of the first and of the second half
            t[0] = (Q[h][0] + Q[h][1] + Q[h][2] + Q[h][3]) * r1;
            t[1] = (Q[h][0] + Q[h][1] - Q[h][2] - Q[h][3]) * r1;
            t[2] = (Q[h][0] - Q[h][1]) * r2;
            t[3] = (Q[h][2] - Q[h][3]) * r2;
            sq[0] = sq[1] = (R[h][0] + R[h][1] + R[h][2] + R[h][3]) * (r1 * r1);
            sq[2] = (R[h][0] + R[h][1]) * (r2 * r2);
            sq[3] = (R[h][2] + R[h][3]) * (r2 * r2);
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              t[k] = Q[h][k];
              sq[k] = R[h][k];
            }
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) corr[h][k] = fmaf(mv, fmaf(t[k], t[k], -sq[k]), corr[h][k]);
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < NS; ++h)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (l0 + k >= L) corr[h][k] = 0.f;
  return cmax;
}

// The shared-source corrections of every coefficient of the leading planes
// added to the variances in bufA (plane rows, buffer offsets vbuf), two
// coefficients per lane and four planes per pass.
template <int D>
__device__ __forceinline__ int shared_source_planes(const DGeom &g, int n, int lane, const int *__restrict__ mem,
                                                    const int *__restrict__ vreg, const int *__restrict__ vbuf,
                                                    const int *__restrict__ vcrd, const float *__restrict__ Sg,
                                                    float *__restrict__ bufA, int MS, const float *mats,
                                                    const int *moff, const float *tab) {
  const int L = min(g.kex, n);
  int cmax = 1;
  for (int s0 = 0; 32 * s0 < g.P; s0 += 2)
    for (int l0 = 0; l0 < L; l0 += 4) {
      float corr[2][4];
      cmax = max(cmax, shared_source_pass<D, 2>(g, n, lane, s0, l0, mem, vreg, vcrd, Sg, mats, moff, tab, corr));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = 32 * (s0 + h) + lane;
        if (q < g.P)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (l0 + k < L) bufA[(l0 + k) * MS + vbuf[q]] += corr[h][k];
      }
    }
  return cmax;
}

// Entry (l, m) of the group-axis transform in double precision (rows as in
// group_axis_entry).
// 1 / sqrt(2^t): 2^(-t/2), times 1/sqrt(2) for odd t (n and b are powers
// of two for the Haar transform).
__device__ __forceinline__ double inv_sqrt_pow2(int t) {
  const double h = ldexp(1.0, -(t >> 1));
  return (t & 1) ? h * 0.70710678118654752440 : h;
}

__device__ __forceinline__ double group_axis_entry64(const DGeom &g, int n, int l, int m) {
  if (g.gtrans != 0) return __ldg(g.dct64 + gen_off(n) + l * n + m);
  const int tn = 31 - __clz(n);
  if (l == 0) return inv_sqrt_pow2(tn);
  const int s = 31 - __clz(l);
  const int b = n >> s, r = l - (1 << s);
  if (m < r * b || m >= (r + 1) * b) return 0.0;
  const double v = inv_sqrt_pow2(tn - s);
  return m < r * b + b / 2 ? v : -v;
}

// Hard-threshold decision (Eq. hard-threshold) for coefficient k = (l, q) of
// a stage-1 group in double precision, for the coefficients whose FP32
// values lie too close to the threshold to decide: Y_k = sum_i T_ki y_i and
// sigma_k^2 = sum_i T_ki^2 m_v(u_i) (Lemma "Covariance propagation", Def.
// "Poisson variance map"), T_ki = A0[l][m] prod_d DCT_d[q_d][p_d] for entry
// i = (member m, patch entry p); for the leading k_ex planes the
// shared-source terms of Def. "Partial shared-source Poisson variance model"
// are added member pair by member pair (as shared_source_planes does);
// Gaussian noise: sigma_k^2 = sigma^2 (Cor. "White-noise transform
// variance").  Keeps Y_k iff |Y_k| > lambda sigma_k; two sides equal to a
// relative 1e-12 are an exact tie in real arithmetic and are not kept.
// mem: member origins (region offsets), vreg: entry offsets, Sg: the staged
// observation.  One lane, sequential; the caller counts it.
__device__ __noinline__ bool ht_keep64(const DGeom &g, int n, int l, int q, const int *__restrict__ mem,
                                       const int *__restrict__ vreg, const float *__restrict__ Sg) {
  const int D = g.D;
  int qc[KMAXD];
  {
    int r = q;
    for (int d = D - 1; d >= 0; --d) {
      qc[d] = r % g.j[d];
      r /= g.j[d];
    }
  }
  auto basis = [&](int p) {
    double f = 1.0;
    for (int d = D - 1; d >= 0; --d) {
      const int J = g.j[d];
      f *= __ldg(g.sp64 + gen_off(J) + qc[d] * J + p % J);
      p /= J;
    }
    return f;
  };
  double Y = 0.0, V = 0.0;
  for (int m = 0; m < n; ++m) {
    const double a = group_axis_entry64(g, n, l, m);
    if (a == 0.0) continue;
    double ys = 0.0, vs = 0.0;
    for (int p = 0; p < g.P; ++p) {
      const double f = basis(p);
      const double y = Sg[mem[m] + vreg[p]];
      ys = fma(f, y, ys);
      if (g.poisson) vs = fma(f * f, g.s_p64 * (y > 0.0 ? y : 0.0), vs);
      else if (g.spatial) vs = fma(f * f, g.var64, vs);
    }
    Y = fma(a, ys, Y);
    V = fma(a * a, vs, V);
  }
  if (!g.poisson) {
    // white noise: sigma^2 (orthonormal) or sigma^2 sum_i T_ki^2 (bior1.5)
    if (!g.spatial) V = g.var64;
  } else if (l < g.kex) {
    for (int m = 0; m < n; ++m) {
      const double am = group_axis_entry64(g, n, l, m);
      if (am == 0.0) continue;
      int cm[KMAXD];
      for (int d = 0; d < D; ++d) cm[d] = (mem[m] / g.rst[d]) % g.RGP[d];
      for (int m2 = m + 1; m2 < n; ++m2) {
        const double am2 = group_axis_entry64(g, n, l, m2);
        if (am2 == 0.0) continue;
        int dl[KMAXD], ext[KMAXD], cnt = 1;
        for (int d = 0; d < D; ++d) {
          dl[d] = (mem[m2] / g.rst[d]) % g.RGP[d] - cm[d];
          ext[d] = g.j[d] - abs(dl[d]);
          cnt *= ext[d] > 0 ? ext[d] : 0;
        }
        double X = 0.0;
        for (int e = 0; e < cnt; ++e) {
          int r = e, off = mem[m];
          double f1 = 1.0, f2 = 1.0;
          for (int d = D - 1; d >= 0; --d) {
            const int pd = (dl[d] > 0 ? dl[d] : 0) + r % ext[d];
            r /= ext[d];
            const int J = g.j[d];
            f1 *= __ldg(g.sp64 + gen_off(J) + qc[d] * J + pd);
            f2 *= __ldg(g.sp64 + gen_off(J) + qc[d] * J + pd - dl[d]);
            off += pd * g.rst[d];
          }
          const double y = Sg[off];
          X = fma(f1 * f2, g.s_p64 * (y > 0.0 ? y : 0.0), X);
        }
        V = fma(2.0 * am * am2, X, V);
      }
    }
  }
  const double t = g.lambda64 * sqrt(V > 0.0 ? V : 0.0);
  return fabs(Y) - t > 1e-12 * t;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ht_keep64 with the warp's lanes sharing the group's entries (and, for the
// shared-source planes, its member pairs); every lane calls it with the same
// (l, q) and gets the same decision.
__device__ __noinline__ bool ht_keep64_warp(const DGeom &g, int n, int l, int q, const int *__restrict__ mem,
                                            const int *__restrict__ vreg, const float *__restrict__ Sg, int lane) {
  const int D = g.D;
  int qc[KMAXD];
  {
    int r = q;
    for (int d = D - 1; d >= 0; --d) {
      qc[d] = r % g.j[d];
      r /= g.j[d];
    }
  }
  double Y = 0.0, V = 0.0;
  const int tot = n * g.P;
  for (int e = lane; e < tot; e += 32) {
    const int m = e / g.P, p = e - m * g.P;
    const double a = group_axis_entry64(g, n, l, m);
    if (a == 0.0) continue;
    double f = a;
    for (int d = D - 1, r = p; d >= 0; --d) {
      const int J = g.j[d];
      f *= __ldg(g.sp64 + gen_off(J) + qc[d] * J + r % J);
      r /= J;
    }
    const double y = Sg[mem[m] + vreg[p]];
    Y = fma(f, y, Y);
    if (g.poisson) V = fma(f * f, g.s_p64 * (y > 0.0 ? y : 0.0), V);
    else if (g.spatial) V = fma(f * f, g.var64, V);
  }
  if (g.poisson && l < g.kex) {
    // shared-source terms, member pairs over the lanes
    for (int t = lane; t < n * n; t += 32) {
      const int m = t / n, m2 = t - m * n;
      if (m2 <= m) continue;
      const double am = group_axis_entry64(g, n, l, m), am2 = group_axis_entry64(g, n, l, m2);
      if (am == 0.0 || am2 == 0.0) continue;
      int dl[KMAXD], ext[KMAXD], cnt = 1;
      for (int d = 0; d < D; ++d) {
        dl[d] = (mem[m2] / g.rst[d]) % g.RGP[d] - (mem[m] / g.rst[d]) % g.RGP[d];
        ext[d] = g.j[d] - abs(dl[d]);
        cnt *= ext[d] > 0 ? ext[d] : 0;
      }
      double X = 0.0;
      for (int e = 0; e < cnt; ++e) {
        int r = e, off = mem[m];
        double f1 = 1.0, f2 = 1.0;
        for (int d = D - 1; d >= 0; --d) {
          const int pd = (dl[d] > 0 ? dl[d] : 0) + r % ext[d];
          r /= ext[d];
          const int J = g.j[d];
          f1 *= __ldg(g.sp64 + gen_off(J) + qc[d] * J + pd);
          f2 *= __ldg(g.sp64 + gen_off(J) + qc[d] * J + pd - dl[d]);
          off += pd * g.rst[d];
        }
        const double y = Sg[off];
        X = fma(f1 * f2, g.s_p64 * (y > 0.0 ? y : 0.0), X);
      }
      V = fma(2.0 * am * am2, X, V);
    }
  }
  Y = warp_sum_d(Y);
  V = warp_sum_d(V);
  // white noise: sigma^2 for an orthonormal transform, sigma^2 sum_i T_ki^2
  // for bior1.5 (Lemma "Covariance propagation")
  if (!g.poisson && !g.spatial) V = g.var64;
  const double t = g.lambda64 * sqrt(V > 0.0 ? V : 0.0);
  return fabs(Y) - t > 1e-12 * t;
}

// FP32 hard-threshold decision with its error band: |X| > lambda sigma is
// taken in FP32 unless |X^2 - lambda^2 s2| lies within the error the FP32
// transforms can carry (eX = 2^-19 ||y_g|| on a coefficient, eS = 2^-20
// (s2 + sum m_v max T^2) on a variance: eight and thirty-two times the
// largest errors of the butterfly DCT and Haar measured against double
// precision on count data, 2^-22 and 2^-25), where the double-precision
// evaluation decides.  Returns 1 keep, 0 drop, -1 undecided in FP32.
__device__ __forceinline__ int ht_decide32(float X, float s2, float lam2, float eX, float eS0) {
  const float xx = X * X, ts = lam2 * s2;
  const float eS = 9.537e-7f * s2 + eS0;
  const float band = 2.f * fabsf(X) * eX + eX * eX + lam2 * eS + 2.5e-7f * (xx + ts);
  if (fabsf(xx - ts) <= band) return -1;
  return xx > ts ? 1 : 0;
}

// Entries (m, v) of a group, m < n members, v < P patch entries, visited with
// a lane stride of 32 and no integer division.
#define BMND_FOR_ENTRIES(body)                         \
  {                                                    \
    int m = lane / P, v = lane - (lane / P) * P;       \
    while (m < n) {                                    \
      body;                                            \
      v += 32;                                         \
      while (v >= P) { v -= P; ++m; }                  \
    }                                                  \
  }

// Lean gathers: entry (m, v) of the group from global arrays at
// gb[m] + vgl[v], GGB independent loads in flight per lane, each value handed
// to put(m, v, a[.], b[.]) (b may be null).
constexpr int GGB = 8;
template <typename Put>
__device__ __forceinline__ void gather_global(const float *__restrict__ a, const float *__restrict__ b,
                                              const int64_t *__restrict__ gb, const int64_t *__restrict__ vgl,
                                              int n, int P, int lane, Put put) {
  int m = lane / P, v = lane - (lane / P) * P;
  while (m < n) {
    float va[GGB], vb[GGB];
    int m1 = m, v1 = v;
#pragma unroll
    for (int k = 0; k < GGB; ++k) {
      va[k] = vb[k] = 0.f;
      if (m1 < n) {
        const int64_t u = gb[m1] + vgl[v1];
        va[k] = __ldg(a + u);
        if (b) vb[k] = __ldg(b + u);
      }
      v1 += 32;
      while (v1 >= P) { v1 -= P; ++m1; }
    }
#pragma unroll
    for (int k = 0; k < GGB; ++k) {
      if (m < n) put(m, v, va[k], vb[k]);
      v += 32;
      while (v >= P) { v -= P; ++m; }
    }
  }
}

// Correction of one group for the second mass-conservation sweep (Def.
// "Aggregation-aware constant-synthesis correction"): zeta = w omega / eta,
// d_g = zeta^T (y_g - p_g), and the sweep adds alpha = d_g / zeta^T 1 to
// every synthesized entry.  p_g: syn[m * MS + vbuf[v]] (vbuf null: column v).
// Entries are visited lane + 32 k in (member, entry) order on every path.
// Out of line: only the second sweep takes it.
template <int D, int PC>
__device__ __noinline__ float mc_alpha(const DGeom &g, int n, int lane, const int *__restrict__ mem,
                                          const int *__restrict__ vreg, const int *__restrict__ vbuf,
                                          const float *__restrict__ omega, const float *__restrict__ wts,
                                          const float *__restrict__ syn, int MS, const float *__restrict__ Sy,
                                          const float *__restrict__ Se, const float *__restrict__ gy,
                                          const float *__restrict__ ge, const int64_t *__restrict__ gb,
                                          const int64_t *__restrict__ vgl, bool lean) {
  const int P = PC ? PC : g.P;
  float dg = 0.f, z1 = 0.f;
  auto term = [&](int m, int v, float et, float yv) {
    const float z = et > 0.f ? wts[m] * omega[v] / et : 0.f;
    dg = fmaf(z, yv - syn[m * MS + (vbuf ? vbuf[v] : v)], dg);
    z1 += z;
  };
  if (D >= 3 && lean) {
    gather_global(ge, gy, gb, vgl, n, P, lane, term);
  } else {
    int m = lane / P, v = lane - (lane / P) * P;
    while (m < n) {
      const int u = mem[m] + vreg[v];
      term(m, v, Se[u], Sy[u]);
      v += 32;
      while (v >= P) { v -= P; ++m; }
    }
  }
  dg = warp_sum(dg);
  z1 = warp_sum(z1);
  return z1 > 0.f ? dg / z1 : 0.f;
}

// Aggregation weight sum of member `lane` from the plane sums r_l in rr_s:
// group scope sum_l r_l, or patch scope sum_l |V_jl|^2 r_l with
// the group-axis DCT.  Out of line: the Haar patch scope is the common case.
__device__ __noinline__ float group_weight_sum(const DGeom &g, int n, int lane, const float *rr_s,
                                               const float *__restrict__ tab) {
  float R = 0.f;
  if (g.wscope == 1) {
    for (int l = 0; l < n; ++l) R += rr_s[l];
  } else {
    const float *Mt = tab + gen_off(n);
    for (int l = 0; l < n; ++l) {
      const float c = __ldg(Mt + l * n + lane);
      R += c * c * rr_s[l];
    }
  }
  return R;
}

// Stage-1 soft thresholding (Eq. soft-threshold) of the group coefficients
// in bufB (variances in bufA when varT, else var_g), as an attenuation
// att = [|X| - lambda sigma]_+ / |X|: bufB receives att X, bufA the weight
// term att^2 (times sigma^2 unless wmodel is 0).  Out of line: inlined beside
// the hard threshold it costs the stage kernels registers.
__device__ __noinline__ void soft_threshold_group(int n, int P, int MS, int lane, const int *__restrict__ vbuf,
                                                  float *bufA, float *bufB, bool varT, float var_g, float lambda,
                                                  int wmodel) {
  BMND_FOR_ENTRIES({
    const int a = m * MS + vbuf[v];
    const float X = bufB[a];
    const float s2 = varT ? bufA[a] : var_g;
    const float ax = fabsf(X);
    const float t = lambda * sqrtf(s2);
    const float att = ax > t ? (ax - t) / ax : 0.f;
    bufB[a] = att * X;
    bufA[a] = att * att * (wmodel == 0 ? 1.f : s2);
  });
}

// Windowed synthesis weights (Def. "Windowed synthesis metrics"): every
// weight term in bufA times the diagonal factor of its spatial coefficient.
__device__ __noinline__ void windowed_weight_terms(const DGeom &g, int n, int P, int MS, int lane,
                                                   const int *__restrict__ vbuf, float *bufA) {
  BMND_FOR_ENTRIES({
    const int a = m * MS + vbuf[v];
    bufA[a] *= syn_energy(g, v);
  });
}

// Settles the hard-threshold coefficients that FP32 left undecided in the
// shared-memory filter (lane L's visit k is entry L + 32 k; the coefficient
// is still in bufB, kept): each decided in double precision by the whole
// warp; those below the threshold and their weight terms go to zero.
__device__ __noinline__ void smem_ht_settle(const DGeom &g, int n, int P, int MS, int lane,
                                            unsigned long long undecided, const int *__restrict__ mem,
                                            const int *__restrict__ vreg, const int *__restrict__ vbuf,
                                            const float *__restrict__ Sg, float *bufA, float *bufB) {
  __syncwarp();
  unsigned pending = __ballot_sync(0xffffffffu, undecided != 0ull);
  while (pending) {
    const int L = __ffs(pending) - 1;
    pending &= pending - 1;
    const unsigned long long um = __shfl_sync(0xffffffffu, undecided, L);
    for (unsigned long long u = um; u; u &= u - 1) {
      const int k = __ffsll((long long)u) - 1;
      const int e = L + 32 * k, m = e / P, v = e - m * P;
      const bool keep = ht_keep64_warp(g, n, m, v, mem, vreg, Sg, lane);
      if (!keep && lane == 0) {
        const int a = m * MS + vbuf[v];
        bufB[a] = 0.f;
        bufA[a] = 0.f;
      }
    }
  }
  if (g.diag) {
    const int t = warp_sum_i(__popcll(undecided));
    if (lane == 0) atomicAdd(g.diag + 2, (unsigned long long)t);
  }
}

// Filters the group whose member origins (region offsets) are in mem[0..n).
// Stage 1: hard thresholding of T y_g against sigma_k from the variance map;
// stage 2: Wiener shrinkage of T y_g with gains from the pilot group.  Leaves
// the synthesized patches in bufB (returns 0) or bufA (returns 1), the patch
// weights in wts, and for the second mass-conservation sweep the correction
// alpha = d_g / (zeta^T 1) of Def. "Aggregation-aware constant-synthesis
// correction" in *alpha_out.
template <int D, int JC, int ST>
__device__ __forceinline__ int filter_group(const DGeom &g, int n, bool mc2, int lane, const int *__restrict__ mem,
                                         const int *__restrict__ vreg, const int *__restrict__ vbuf,
                                         const float *__restrict__ omega, const float *__restrict__ Sg,
                                         const float *__restrict__ Sy, const float *__restrict__ Se,
                                         float *__restrict__ bufA, float *__restrict__ bufB, float *__restrict__ wts,
                                         float *__restrict__ rr_s, const float *mats, const int *moff,
                                         const int *__restrict__ vcrd, const float *tab,
                                         const float *__restrict__ gy,
                                         const float *__restrict__ ge, const int64_t *__restrict__ gb,
                                         const int64_t *__restrict__ vgl, float *alpha_out,
                                         unsigned long long *diag) {
  using SH = CubeShape<D, JC>;
  const int P = SH::fixed ? SH::P : g.P;
  const int MS = SH::fixed ? SH::MS : g.MS;
  const bool stage2 = ST ? ST == 2 : g.stage == 2;  // ST: stage fixed at compile time
  // The transforms run as one loop over a short phase list so that the
  // transform code is inlined once: before each transform, the phase's own
  // gather / shrink / gain step.
  //   stage 1: T^2 m_v (Poisson) | T y_g | shrink, weights | T^T C
  //   stage 2: T^2 m_v (Poisson) | T gamma_g | gains, weights | T y_g | G Y, T^T C
  const float lam2 = g.lambda * g.lambda;
  float *syn = stage2 ? bufA : bufB;
  // coefficient variances by the squared transform: Poisson noise, and white
  // noise under the non-orthonormal bior1.5 (sigma^2 sum_i T_ki^2); else
  // sigma^2 itself (Cor. "White-noise transform variance")
  const bool varT = g.poisson || g.spatial;
  const int first = varT ? 0 : 1;
  const int last = stage2 ? 4 : 3;
  // stage-1 hard threshold: group norm and variance-map total for the FP32
  // error band of the decision (ht_decide32)
  const bool hard = !stage2 && !g.soft;
  float n2 = 0.f, sm = 0.f;
  for (int ph = first; ph <= last; ++ph) {
    float *tb;
    int tmode;
    if (ph == 0) {
      // gather the guide group (y in stage 1, pilot in stage 2) and, for
      // Poisson data, its variance map m_v = s_P [guide]_+; then
      // sigma_k^2 = sum_i T_ki^2 m_v(u_i)
      {
        const bool pois = g.poisson;
        const float sp = g.s_p, var_g = g.var_g;
        auto put = [&](int a, float gv) {
          bufB[a] = gv;
          const float mv = pois ? sp * fmaxf(gv, 0.f) : var_g;
          bufA[a] = mv;
          n2 = fmaf(gv, gv, n2);
          sm += mv;
        };
        if constexpr (SH::fixed && SH::P % 32 == 0) {
          // two members' entries loaded before they are stored
          constexpr int KV = SH::P / 32;
          int vb[KV], vr[KV];
#pragma unroll
          for (int k = 0; k < KV; ++k) {
            vb[k] = vbuf[lane + 32 * k];
            vr[k] = vreg[lane + 32 * k];
          }
          for (int m0 = 0; m0 < n; m0 += 2) {
            const bool two = m0 + 1 < n;
            const int o0 = mem[m0], o1 = two ? mem[m0 + 1] : o0;
            float t0[KV], t1[KV];
#pragma unroll
            for (int k = 0; k < KV; ++k) {
              t0[k] = Sg[o0 + vr[k]];
              t1[k] = Sg[o1 + vr[k]];
            }
#pragma unroll
            for (int k = 0; k < KV; ++k) {
              put(m0 * MS + vb[k], t0[k]);
              if (two) put((m0 + 1) * MS + vb[k], t1[k]);
            }
          }
        } else {
          BMND_FOR_ENTRIES(put(m * MS + vbuf[v], Sg[mem[m] + vreg[v]]));
        }
      }
      __syncwarp();
      tb = bufA;
      tmode = 2;
    } else if (ph == 1) {
      if (!varT) {
        BMND_FOR_ENTRIES({
          const float gv = Sg[mem[m] + vreg[v]];
          bufB[m * MS + vbuf[v]] = gv;
          n2 = fmaf(gv, gv, n2);
        });
        __syncwarp();
      }
      tb = bufB;
      tmode = 0;
    } else if (ph == 2) {
      int cmax = 0;
      if (g.kex > 0 && g.poisson) {
        cmax = shared_source_planes<D>(g, n, lane, mem, vreg, vbuf, vcrd, Sg, bufA, MS, mats, moff, tab);
        __syncwarp();
      }
      float eX = 0.f, eS0 = 0.f, eSx = 0.f;
      if (hard) {
        n2 = warp_sum(n2);
        sm = warp_sum(sm);
        const float a2 = n == 1 ? 1.f : (g.gtrans == 0 ? 0.5f : 2.f / (float)n);
        eX = 1.9073e-6f * g.ht_band * sqrtf(n2);
        eS0 = 9.537e-7f * g.ht_band * sm * a2 * g.ht_t2;
        // shared-source planes: FP32 error of the per-location terms
        // m_v (t^2 - sum a^2), at most a few ulps per covering member of
        // sum_u m_v sum_i a_i^2 <= a2 max F^2 sum m_v
        eSx = 4.77e-7f * (float)cmax * sm * a2 * g.ht_t2;
      }
      // undecided hard-threshold coefficients of this lane, by visit number
      // (entries lane + 32 k); kept until settled below
      unsigned long long undecided = 0ull;
      int visit = 0;
      // ---- shrinkage; per-coefficient weight terms into bufA.  The
      // profile's scalars are read once: the group buffers share the shared
      // memory with the job descriptor, so the compiler would otherwise
      // reload them after every store ----
      const bool soft = g.soft, wdomain = g.wdomain != 0;
      const int wmodel = g.wmodel, kex = g.kex;
      const float var_g = g.var_g, lambda = g.lambda, a_power = g.a_power, s_v = g.s_v;
      // the shrinkage of coefficient a = (m, v) with value X and variance s2,
      // entry number vis of this lane
      auto shrink = [&](int m, int v, int a, float X, float s2, int vis) {
        float wterm;
        if (!stage2) {
          // |X| > lambda sigma; undecided in FP32: kept until settled
          int kp = ht_decide32(X, s2, lam2, eX, m < kex ? eS0 + eSx : eS0);
          if (kp < 0) {
            // at most 64 visits per lane with compile-time patches of <= 64
            // entries (32 members at most); past 64 visits: at once
            if (vis < 64 || (SH::fixed && SH::P <= 64)) undecided |= 1ull << (vis & 63);
            else kp = ht_keep64(g, n, m, v, mem, vreg, Sg) ? 1 : 0;
          }
          bufB[a] = kp ? X : 0.f;
          wterm = kp ? (wmodel == 0 ? 1.f : s2) : 0.f;
        } else {
          const float S = fmaxf(X * X - a_power * s2, 0.f);
          const float den = S + s_v * s2;
          const float G = den > 0.f ? __fdividef(S, den) : 0.f;
          bufB[a] = G;
          wterm = wmodel == 0 ? G * G : (wmodel == 1 ? G * G * s2 : G * G * s2 + (1.f - G) * (1.f - G) * S);
        }
        bufA[a] = wterm;
      };
      if constexpr (SH::fixed && SH::P % 32 == 0 && ST == 2) {
        // Wiener stage, compile-time patches: this lane's entries v = lane +
        // 32 k of two members are loaded before any of them is written back
        // (the hard-threshold stage keeps one entry at a time: four inlined
        // copies of its decision measured slower)
        constexpr int KV = SH::P / 32;
        int vb[KV];
#pragma unroll
        for (int k = 0; k < KV; ++k) vb[k] = vbuf[lane + 32 * k];
        for (int m0 = 0; m0 < n; m0 += 2) {
          const bool two = m0 + 1 < n;
          float Xv[2][KV], Sv[2][KV];
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < KV; ++k) {
              const int a = (m0 + h) * MS + vb[k];
              const bool in = h == 0 || two;
              Xv[h][k] = in ? bufB[a] : 0.f;
              Sv[h][k] = in && varT ? bufA[a] : var_g;
            }
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int k = 0; k < KV; ++k)
              if (h == 0 || two)
                shrink(m0 + h, lane + 32 * k, (m0 + h) * MS + vb[k], Xv[h][k], Sv[h][k], (m0 + h) * KV + k);
        }
      } else if (!stage2 && soft) {
        soft_threshold_group(n, P, MS, lane, vbuf, bufA, bufB, varT, var_g, lambda, wmodel);
      } else {
        BMND_FOR_ENTRIES({
          const int a = m * MS + vbuf[v];
          shrink(m, v, a, bufB[a], varT ? bufA[a] : var_g, visit);
          ++visit;
        });
      }
      if (hard && __any_sync(0xffffffffu, undecided != 0ull))
        smem_ht_settle(g, n, P, MS, lane, undecided, mem, vreg, vbuf, Sg, bufA, bufB);
      __syncwarp();
      if (wdomain) {
        windowed_weight_terms(g, n, P, MS, lane, vbuf, bufA);
        __syncwarp();
      }
      // ---- r_l = sum_q (term) for every group-axis plane l (lane l sums
      // its row, starting at its own entry so the reads spread over banks;
      // four partial sums, so that the adds do not wait on one another) ----
      if (lane < n) {
        float r0 = 0.f, r1 = 0.f, r2 = 0.f, r3 = 0.f;
        const float *row = bufA + lane * MS;
        int v = lane % P, t = 0;
        for (; t + 4 <= P; t += 4) {
          const int v1 = v + 1 == P ? 0 : v + 1;
          const int v2 = v1 + 1 == P ? 0 : v1 + 1;
          const int v3 = v2 + 1 == P ? 0 : v2 + 1;
          r0 += row[vbuf[v]];
          r1 += row[vbuf[v1]];
          r2 += row[vbuf[v2]];
          r3 += row[vbuf[v3]];
          v = v3 + 1 == P ? 0 : v3 + 1;
        }
        for (; t < P; ++t) {
          r0 += row[vbuf[v]];
          v = v + 1 == P ? 0 : v + 1;
        }
        rr_s[lane] = (r0 + r1) + (r2 + r3);
      }
      __syncwarp();
      // ---- weights: patch scope R_j = sum_l |V_jl|^2 r_l, group scope sum_l r_l
      if (lane < n) {
        float R = 0.f;
        if (g.wscope == 0 && g.gtrans == 0) {
          R = rr_s[0] / (float)n;
          for (int bb = n; bb >= 2; bb >>= 1) R += rr_s[n / bb + lane / bb] / (float)bb;
        } else {
          R = group_weight_sum(g, n, lane, rr_s, tab);
        }
        wts[lane] = R > 0.f ? 1.f / R : 1.f;
      }
      __syncwarp();
      if (stage2) {
        // Wiener: the observation group, to be transformed next
        if (D >= 3 && g.lean)
          gather_global(gy, nullptr, gb, vgl, n, P, lane,
                        [&](int m, int v, float x, float) { bufA[m * MS + vbuf[v]] = x; });
        else if constexpr (SH::fixed && SH::P % 32 == 0) {
          // two members' entries loaded before they are stored
          constexpr int KV = SH::P / 32;
          int vb[KV], vr[KV];
#pragma unroll
          for (int k = 0; k < KV; ++k) {
            vb[k] = vbuf[lane + 32 * k];
            vr[k] = vreg[lane + 32 * k];
          }
          for (int m0 = 0; m0 < n; m0 += 2) {
            const bool two = m0 + 1 < n;
            const int o0 = mem[m0], o1 = two ? mem[m0 + 1] : o0;
            float t0[KV], t1[KV];
#pragma unroll
            for (int k = 0; k < KV; ++k) {
              t0[k] = Sy[o0 + vr[k]];
              t1[k] = Sy[o1 + vr[k]];
            }
#pragma unroll
            for (int k = 0; k < KV; ++k) {
              bufA[m0 * MS + vb[k]] = t0[k];
              if (two) bufA[(m0 + 1) * MS + vb[k]] = t1[k];
            }
          }
        } else {
          BMND_FOR_ENTRIES({ bufA[m * MS + vbuf[v]] = Sy[mem[m] + vreg[v]]; });
        }
        __syncwarp();
        tb = bufA;
        tmode = 0;
      } else {
        tb = bufB;
        tmode = 1;
      }
    } else if (ph == 3) {
      if (stage2) {
        if constexpr (SH::fixed && SH::P % 32 == 0) {
          constexpr int KV = SH::P / 32;
          int vb[KV];
#pragma unroll
          for (int k = 0; k < KV; ++k) vb[k] = vbuf[lane + 32 * k];
          for (int m0 = 0; m0 < n; m0 += 2) {
            const bool two = m0 + 1 < n;
            float x0[KV], x1[KV], g0[KV], g1[KV];
#pragma unroll
            for (int k = 0; k < KV; ++k) {
              const int a0 = m0 * MS + vb[k], a1 = two ? a0 + MS : a0;
              x0[k] = bufA[a0];
              g0[k] = bufB[a0];
              x1[k] = bufA[a1];
              g1[k] = bufB[a1];
            }
#pragma unroll
            for (int k = 0; k < KV; ++k) {
              bufA[m0 * MS + vb[k]] = x0[k] * g0[k];
              if (two) bufA[(m0 + 1) * MS + vb[k]] = x1[k] * g1[k];
            }
          }
        } else {
          BMND_FOR_ENTRIES({
            const int a = m * MS + vbuf[v];
            bufA[a] *= bufB[a];
          });
        }
        __syncwarp();
        tb = bufA;
        tmode = 1;
      } else {
        break;
      }
    } else {
      break;
    }
    group_xform<D, JC>(tb, g, n, tmode, lane, vbuf, mats, moff, tab);
  }
  float alpha = 0.f;
  if (mc2)
    alpha = mc_alpha<D, 0>(g, n, lane, mem, vreg, vbuf, omega, wts, syn, MS, Sy, Se, gy, ge, gb, vgl, g.lean);
  *alpha_out = alpha;
  return stage2 ? 1 : 0;
}

// ---------------------------------------------------------------------------
// group filter with register-resident patches (cubic patches, P <= 64, Haar)
// ---------------------------------------------------------------------------
// Group buffers are [member][MS] with MS = P | 1 (odd), entry v in column v:
// a lane reading one member's row and a lane reading one entry's column both
// touch 32 distinct banks.  Row phases (lane = member) run the separable
// patch DCT in registers; column phases (lane = entry) run the Haar along the
// group axis in registers together with the shrinkage it feeds.

// Column of entry v: y_m = buf[m * MS + v] for m < N.
template <int N, int MS>
__device__ __forceinline__ void col_load(float (&y)[N], const float *buf, int v) {
#pragma unroll
  for (int m = 0; m < N; ++m) y[m] = buf[m * MS + v];
}
template <int N, int MS>
__device__ __forceinline__ void col_store(float *buf, int v, const float (&y)[N]) {
#pragma unroll
  for (int m = 0; m < N; ++m) buf[m * MS + v] = y[m];
}

// Shared-source corrections of the leading group-axis planes (column of
// the register filter; cx holds planes 0..3, zero beyond k_ex).
template <int N>
__device__ __forceinline__ void add_shared_source(float (&S)[N], float4 cx) {
  const float c[4] = {cx.x, cx.y, cx.z, cx.w};
#pragma unroll
  for (int m = 0; m < (N < 4 ? N : 4); ++m) S[m] += c[m];
}

// Stage 1, one column: sigma^2 = H^2 s (s = T_patch^2 m_v in bufA, or the
// Gaussian variance), X = H x, hard threshold with weight terms into bufA,
// then H^T of the kept coefficients back into bufB.
// Returns the planes whose hard-threshold decision FP32 cannot take
// (bitmask); they are kept for now and settled by col_ht_settle.
template <int N, int MS>
__device__ __forceinline__ unsigned col_hard_threshold(const DGeom &g, float *bufA, float *bufB, int v, float lam2,
                                                       float eX, float eS0, float4 cx, float eSx) {
  unsigned undecided = 0u;
  float X[N], S[N];
  col_load<N, MS>(X, bufB, v);
  haar_fwd_levels<N, N, false>(X);
  if (g.poisson) {
    col_load<N, MS>(S, bufA, v);
    haar_fwd_levels<N, N, true>(S);
    add_shared_source<N>(S, cx);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) S[m] = g.var_g;
  }
#pragma unroll
  for (int m = 0; m < N; ++m) {
    // |X| > lambda sigma; undecided in FP32: kept until col_ht_settle
    const int kp = ht_decide32(X[m], S[m], lam2, eX, m < g.kex ? eS0 + eSx : eS0);
    if (kp < 0) undecided |= 1u << m;
    bufA[m * MS + v] = kp ? (g.wmodel == 0 ? 1.f : S[m]) : 0.f;
    X[m] = kp ? X[m] : 0.f;
  }
  haar_inv_levels<N, 2>(X);
  col_store<N, MS>(bufB, v, X);
  return undecided;
}

// Stage 1 with soft thresholding, one column (as col_hard_threshold): Eq.
// (soft-threshold) as an attenuation att = [|X| - lambda sigma]_+ / |X|,
// weight terms |att|^2 (times sigma^2).  Out of line: inlined beside the
// hard threshold it costs the stage kernels registers.
template <int N, int MS>
__device__ __noinline__ void col_soft_threshold(const DGeom &g, float *bufA, float *bufB, int v, float4 cx) {
  float X[N], S[N];
  col_load<N, MS>(X, bufB, v);
  haar_fwd_levels<N, N, false>(X);
  if (g.poisson) {
    col_load<N, MS>(S, bufA, v);
    haar_fwd_levels<N, N, true>(S);
    add_shared_source<N>(S, cx);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) S[m] = g.var_g;
  }
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const float ax = fabsf(X[m]), t = g.lambda * sqrtf(S[m]);
    const float att = ax > t ? (ax - t) / ax : 0.f;
    bufA[m * MS + v] = att * att * (g.wmodel == 0 ? 1.f : S[m]);
    X[m] = att * X[m];
  }
  haar_inv_levels<N, 2>(X);
  col_store<N, MS>(bufB, v, X);
}

// Drops the planes in `drop` from the stored column v (H^T of the kept
// coefficients): forward Haar, zero, inverse Haar; their weight terms go to
// zero.
template <int N, int MS>
__device__ __forceinline__ void col_ht_drop(float *bufA, float *bufB, int v, unsigned drop) {
  float X[N];
  col_load<N, MS>(X, bufB, v);
  haar_fwd_levels<N, N, false>(X);
#pragma unroll
  for (int m = 0; m < N; ++m)
    if (drop & (1u << m)) {
      X[m] = 0.f;
      bufA[m * MS + v] = 0.f;
    }
  haar_inv_levels<N, 2>(X);
  col_store<N, MS>(bufB, v, X);
}

// Stage 2, one column: sigma^2 as above from the pilot, Gamma = H gamma,
// Wiener gains G into bufB and weight terms into bufA.
template <int N, int MS>
__device__ __forceinline__ void col_wiener_gain(const DGeom &g, float *bufA, float *bufB, int v, float4 cx) {
  float X[N], S[N];
  col_load<N, MS>(X, bufB, v);
  haar_fwd_levels<N, N, false>(X);
  if (g.poisson) {
    col_load<N, MS>(S, bufA, v);
    haar_fwd_levels<N, N, true>(S);
    add_shared_source<N>(S, cx);
  } else {
#pragma unroll
    for (int m = 0; m < N; ++m) S[m] = g.var_g;
  }
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const float s2 = S[m];
    const float Sx = fmaxf(X[m] * X[m] - g.a_power * s2, 0.f);
    const float den = Sx + g.s_v * s2;
    const float G = den > 0.f ? __fdividef(Sx, den) : 0.f;
    bufB[m * MS + v] = G;
    bufA[m * MS + v] = g.wmodel == 0 ? G * G
                                     : (g.wmodel == 1 ? G * G * s2 : G * G * s2 + (1.f - G) * (1.f - G) * Sx);
  }
}

// Stage 2, one column: Y = H y, C = G Y, H^T C back into bufA.
template <int N, int MS>
__device__ __forceinline__ void col_wiener_apply(float *bufA, const float *bufB, int v) {
  float Y[N];
  col_load<N, MS>(Y, bufA, v);
  haar_fwd_levels<N, N, false>(Y);
#pragma unroll
  for (int m = 0; m < N; ++m) Y[m] *= bufB[m * MS + v];
  haar_inv_levels<N, 2>(Y);
  col_store<N, MS>(bufA, v, Y);
}

// Runs the column operation OP(N) for the lane's entries, N = n.
#define BMND_COLUMNS(OP)                                             \
  for (int v = lane; v < P; v += 32) {                               \
    switch (n) {                                                     \
      case 1: OP(1); break;                                          \
      case 2: OP(2); break;                                          \
      case 4: OP(4); break;                                          \
      case 8: OP(8); break;                                          \
      case 16: OP(16); break;                                        \
      default: OP(32); break;                                        \
    }                                                                \
  }

// Settles the hard-threshold coefficients that FP32 left undecided in the
// register filter (one column per lane, `undecided` the lane's planes; they
// were kept): each decided in double precision by the whole warp, and the
// columns of those below the threshold redone without them.
template <int MS>
__device__ __noinline__ void rf_ht_settle(const DGeom &g, int n, int lane, unsigned undecided,
                                          const int *__restrict__ mem, const int *__restrict__ vreg,
                                          const float *__restrict__ Sg, float *bufA, float *bufB) {
  unsigned pending = __ballot_sync(0xffffffffu, undecided != 0u);
  unsigned drop = 0u;
  while (pending) {
    const int L = __ffs(pending) - 1;
    pending &= pending - 1;
    for (unsigned u = __shfl_sync(0xffffffffu, undecided, L); u; u &= u - 1) {
      const int m = __ffs(u) - 1;
      const bool keep = ht_keep64_warp(g, n, m, L, mem, vreg, Sg, lane);
      if (!keep && lane == L) drop |= 1u << m;
    }
  }
  if (drop) {
    const int v = lane;
    switch (n) {
      case 1: col_ht_drop<1, MS>(bufA, bufB, v, drop); break;
      case 2: col_ht_drop<2, MS>(bufA, bufB, v, drop); break;
      case 4: col_ht_drop<4, MS>(bufA, bufB, v, drop); break;
      case 8: col_ht_drop<8, MS>(bufA, bufB, v, drop); break;
      case 16: col_ht_drop<16, MS>(bufA, bufB, v, drop); break;
      default: col_ht_drop<32, MS>(bufA, bufB, v, drop); break;
    }
  }
  if (g.diag) {
    const int t = warp_sum_i(__popc(undecided));
    if (lane == 0) atomicAdd(g.diag + 2, (unsigned long long)t);
  }
}

template <int D, int JC, int ST>
__device__ __forceinline__ int filter_group_rf(const DGeom &g, int n, bool mc2, int lane, const int *__restrict__ mem,
                                            const int *__restrict__ vreg, const float *__restrict__ omega,
                                            const float *__restrict__ Sg, const float *__restrict__ Sy,
                                            const float *__restrict__ Se, float *__restrict__ bufA,
                                            float *__restrict__ bufB, float *__restrict__ wts,
                                            float *__restrict__ rr_s, const float *__restrict__ gy,
                                            const float *__restrict__ ge, const int64_t *__restrict__ gb,
                                            const int64_t *__restrict__ vgl, float *alpha_out,
                                            unsigned long long *diag, const float *mats, const int *moff,
                                            const int *__restrict__ vcrd, const float *tab) {
  constexpr int P = ipow(JC, D);
  constexpr int MS = CubeShape<D, JC>::MS;
  static_assert(MS == (P | 1), "register filter layout");
  const bool stage2 = ST ? ST == 2 : g.stage == 2;  // ST: stage fixed at compile time
  // ---- entries of a shared region into rows of buf (lanes over entries)
  auto gather = [&](float *buf, const float *src) {
    if constexpr (P % 32 == 0) {
      constexpr int KV = P / 32;
      int vr[KV];
#pragma unroll
      for (int k = 0; k < KV; ++k) vr[k] = vreg[lane + 32 * k];
      for (int m = 0; m < n; ++m) {
        const float *s0 = src + mem[m];
#pragma unroll
        for (int k = 0; k < KV; ++k) buf[m * MS + lane + 32 * k] = s0[vr[k]];
      }
    } else {
      const int v = lane % P, vr = vreg[v];
      for (int m = lane / P; m < n; m += 32 / P) buf[m * MS + v] = src[mem[m] + vr];
    }
  };
  // ---- row phases: one member per lane, the patch DCT in registers
  auto row_dct = [&](float *buf, auto mode) {
    if (lane < n) {
      float x[P];
      float *row = buf + lane * MS;
#pragma unroll
      for (int i = 0; i < P; ++i) x[i] = row[i];
      dct_patch<D, JC, decltype(mode)::value>(x);
#pragma unroll
      for (int i = 0; i < P; ++i) row[i] = x[i];
    }
  };
  using F = std::integral_constant<int, 0>;
  using I = std::integral_constant<int, 1>;
  // guide group into bufB; for Poisson data also T_patch^2 m_v into bufA
  gather(bufB, Sg);
  __syncwarp();
  // stage-1 hard threshold: group norm and variance-map total (s_P times
  // the positive part of y_g) for the FP32 error band of the decision
  // (ht_decide32), from the gathered values
  // partial shared-source variance of the leading planes (at most 4 here):
  // corrections of this lane's column, added after the squared group-axis
  // Haar; eSx widens their FP32 band (as in filter_group)
  float4 cx = make_float4(0.f, 0.f, 0.f, 0.f);
  int cmax = 0;
  if (g.kex > 0 && g.poisson) {
    float corr[1][4];
    cmax = shared_source_pass<D, 1>(g, n, lane, 0, 0, mem, vreg, vcrd, Sg, mats, moff, tab, corr);
    cx = make_float4(corr[0][0], corr[0][1], corr[0][2], corr[0][3]);
  }
  float eX = 0.f, eS0 = 0.f, eSx = 0.f;
  if (!stage2 && !g.soft) {
    float n2 = 0.f, sm = 0.f;
    for (int e = lane; e < n * P; e += 32) {
      const float gv = bufB[(e / P) * MS + e % P];
      n2 = fmaf(gv, gv, n2);
      sm += fmaxf(gv, 0.f);
    }
    n2 = warp_sum(n2);
    eX = 1.9073e-6f * sqrtf(n2);
    if (g.poisson) {
      sm = warp_sum(sm) * g.s_p;
      const float a2 = n == 1 ? 1.f : 0.5f;
      eS0 = 9.537e-7f * sm * a2 * g.ht_t2;
      eSx = 4.77e-7f * (float)cmax * sm * a2 * g.ht_t2;
    }
  }
  if (g.poisson && lane < n) {
    float x[P];
    const float *row = bufB + lane * MS;
#pragma unroll
    for (int i = 0; i < P; ++i) x[i] = g.s_p * fmaxf(row[i], 0.f);
    dct_patch<D, JC, 2>(x);
    float *out = bufA + lane * MS;
#pragma unroll
    for (int i = 0; i < P; ++i) out[i] = x[i];
  }
  row_dct(bufB, F{});
  __syncwarp();
  if (!stage2) {
    const float lam2 = g.lambda * g.lambda;
    // one column per lane (P <= 32): the undecided planes of column `lane`
    if (g.soft) {
#define BMND_OP(NN) col_soft_threshold<NN, MS>(g, bufA, bufB, v, cx)
      BMND_COLUMNS(BMND_OP)
#undef BMND_OP
    } else {
      unsigned undecided = 0u;
#define BMND_OP(NN) undecided = col_hard_threshold<NN, MS>(g, bufA, bufB, v, lam2, eX, eS0, cx, eSx)
      BMND_COLUMNS(BMND_OP)
#undef BMND_OP
      if (__any_sync(0xffffffffu, undecided != 0u))
        rf_ht_settle<MS>(g, n, lane, undecided, mem, vreg, Sg, bufA, bufB);
    }
  } else {
#define BMND_OP(NN) col_wiener_gain<NN, MS>(g, bufA, bufB, v, cx)
    BMND_COLUMNS(BMND_OP)
#undef BMND_OP
  }
  __syncwarp();
  // ---- r_l = sum_q (term) for every group-axis plane l (windowed
  // synthesized domain: each term times the metric factor of its spatial
  // coefficient, the per-axis product at compile-time coordinates); weights
  if (lane < n) {
    float r = 0.f;
    const float *row = bufA + lane * MS;
    if (g.wdomain) {
#pragma unroll
      for (int v = 0; v < P; ++v) {
        float e = 1.f;
#pragma unroll
        for (int d = D - 1, rem = v; d >= 0; --d, rem /= JC) e *= g.wsyn[d][rem % JC];
        r = fmaf(e, row[v], r);
      }
    } else {
#pragma unroll
      for (int v = 0; v < P; ++v) r += row[v];
    }
    rr_s[lane] = r;
  }
  __syncwarp();
  if (lane < n) {
    float R = 0.f;
    if (g.wscope == 1) {
      for (int l = 0; l < n; ++l) R += rr_s[l];
    } else {
      // patch scope R_j = sum_l |V_jl|^2 r_l for the Haar basis ordered
      // [scaling, coarsest detail, ..., finest details]
      R = rr_s[0] / (float)n;
      for (int bb = n; bb >= 2; bb >>= 1) R += rr_s[n / bb + lane / bb] / (float)bb;
    }
    wts[lane] = R > 0.f ? 1.f / R : 1.f;
  }
  __syncwarp();
  float *syn;
  if (!stage2) {
    row_dct(bufB, I{});
    syn = bufB;
  } else {
    // Wiener: the observation group, transformed, scaled by G, inverted
    if (D >= 3 && g.lean)
      gather_global(gy, nullptr, gb, vgl, n, P, lane, [&](int m, int v, float x, float) { bufA[m * MS + v] = x; });
    else
      gather(bufA, Sy);
    __syncwarp();
    row_dct(bufA, F{});
    __syncwarp();
#define BMND_OP(NN) col_wiener_apply<NN, MS>(bufA, bufB, v)
    BMND_COLUMNS(BMND_OP)
#undef BMND_OP
    __syncwarp();
    row_dct(bufA, I{});
    syn = bufA;
  }
  __syncwarp();
  float alpha = 0.f;
  if (mc2)
    alpha = mc_alpha<D, P>(g, n, lane, mem, vreg, nullptr, omega, wts, syn, MS, Sy, Se, gy, ge, gb, vgl, g.lean);
  *alpha_out = alpha;
  return stage2 ? 1 : 0;
}

// ---------------------------------------------------------------------------
// the stage kernel
// ---------------------------------------------------------------------------

// Shared-memory layout of one job (the host computes the same sizes).
struct SmemLayout {
  float *bsm;    // stage-1 noise bias: patch sums of the guide per region position
  int *vreg, *vbuf, *rowoff, *moff, *fvoff, *fpreg;
  int *vcrd;     // shared-source variance: patch-entry coordinates, 5 bits per axis
  int64_t *vgl;  // lean: global offset of every patch entry
  float *omega, *mats, *Sg, *Sy, *Se;
  float2 *acc;
  unsigned char *warps;
  int wbytes;
};

__device__ __forceinline__ unsigned char *al16p(unsigned char *p) {
  return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
}

// cached: second mass-conservation sweep from the synthesis cache, which
// stages y and eta (never read from global memory) and no guide, and needs
// one group buffer per warp.
__device__ SmemLayout smem_layout(unsigned char *smem, const DGeom &g, bool stage2, bool mc2, bool cached) {
  SmemLayout s;
  unsigned char *p = smem + ((sizeof(DJob) + 15) & ~(size_t)15);
  s.vreg = reinterpret_cast<int *>(p); p += sizeof(int) * g.P;
  s.vbuf = reinterpret_cast<int *>(p); p += sizeof(int) * g.P;
  s.omega = reinterpret_cast<float *>(p); p += sizeof(float) * g.P;
  s.rowoff = reinterpret_cast<int *>(p); p += sizeof(int) * g.rows;
  s.moff = reinterpret_cast<int *>(p); p += sizeof(int) * KMAXD;
  s.fvoff = reinterpret_cast<int *>(p); p += sizeof(int) * (g.fp ? g.P : 0);
  s.fpreg = reinterpret_cast<int *>(p); p += sizeof(int) * g.fp;
  s.vcrd = reinterpret_cast<int *>(p); p += sizeof(int) * (g.kex ? g.P : 0);
  p = al16p(p);
  s.vgl = reinterpret_cast<int64_t *>(p); p += sizeof(int64_t) * (g.lean ? g.P : 0);
  p = al16p(p);
  s.mats = reinterpret_cast<float *>(p);
  for (int a = 0; a < g.D; ++a) p += sizeof(float) * mat_block(g.j[a]);
  p = al16p(p);
  s.bsm = reinterpret_cast<float *>(p);
  p += sizeof(float) * (g.bsm && !stage2 && !mc2 && !cached ? g.region + RPAD : 0);
  p = al16p(p);
  const int RS = g.region + RPAD;
  s.Sg = reinterpret_cast<float *>(p); p += sizeof(float) * RS;
  s.Sy = s.Sg;
  s.Se = nullptr;
  if (cached) {
    // region 0 holds y, region 1 eta
    s.Se = reinterpret_cast<float *>(p); p += sizeof(float) * RS;
  } else {
    if (stage2 && !g.lean) { s.Sy = reinterpret_cast<float *>(p); p += sizeof(float) * RS; }
    if (mc2 && !g.lean) { s.Se = reinterpret_cast<float *>(p); p += sizeof(float) * RS; }
  }
  p = al16p(p);
  s.acc = reinterpret_cast<float2 *>(p); p += sizeof(float2) * g.region;
  s.warps = al16p(p);
  s.wbytes = cached ? warp_bytes(g.M, g.MS, g.fp, 0, 1) : warp_bytes(g.M, g.MS, g.fp, g.lean);
  return s;
}

// mode 0: match + filter + aggregate (group tables written if job.groups);
// mode 1: match only, group tables written; mode 2: mass-conservation sweep 2
// (groups read back, corrected patches aggregated with the sweep-1 weights).
// Persistent: each CTA takes tiles from *counter until all are done.
// Adds the group's weighted synthesized patches to dst in member order
// (Def. "Weighted overlap-add estimate"): member m's entry v (synthesized
// value syn[m MS + vbuf[v]]) at dst[mbase[m] + eoff[v]], numerator
// w_m omega_v (value + alpha), denominator w_m omega_v; the warp's lanes
// over the entries (distinct locations), one member after another.  PF:
// the patch size when it is a compile-time multiple of 32, else 0.
template <int PF>
__device__ __forceinline__ void add_members_to(float2 *dst, const int *mbase, const int *__restrict__ eoff, int n,
                                               int P, int MS, int lane, const float *syn, const float *wts,
                                               float alpha, const float *__restrict__ omega,
                                               const int *__restrict__ vbuf) {
  if constexpr (PF > 0) {
    constexpr int KV = PF / 32;
    int eo[KV], vb[KV];
    float om[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
      eo[k] = eoff[lane + 32 * k];
      vb[k] = vbuf[lane + 32 * k];
      om[k] = omega[lane + 32 * k];
    }
    for (int m = 0; m < n; ++m) {
      const int b = mbase[m];
      const float wm = wts[m];
      const float *sr = syn + m * MS;
#pragma unroll
      for (int k = 0; k < KV; ++k) {
        const float wo = wm * om[k];
        float2 t = dst[b + eo[k]];
        t.x = fmaf(wo, sr[vb[k]] + alpha, t.x);
        t.y += wo;
        dst[b + eo[k]] = t;
      }
      __syncwarp();
    }
  } else {
    for (int m = 0; m < n; ++m) {
      const int b = mbase[m];
      const float wm = wts[m];
      const float *sr = syn + m * MS;
      for (int v = lane; v < P; v += 32) {
        const float wo = wm * omega[v];
        float2 t = dst[b + eoff[v]];
        t.x = fmaf(wo, sr[vbuf[v]] + alpha, t.x);
        t.y += wo;
        dst[b + eoff[v]] = t;
      }
      __syncwarp();
    }
  }
}

// Private footprint of one reference (local index rl in its tile): the box
// [core, core + 2 rad + j - 1] holds every member patch; lvl[m] receives
// member m's offset in the box, the box (fpb, g.fp entries) the group's
// weighted patches.  Returns the box's offset in the tile region.  Out of
// line: inlined it costs the stage kernels registers.
template <int D, int PF>
__device__ __noinline__ int fp_export(const DGeom &g, int rl, int n, int P, int MS, int lane, const int *mem,
                                      int *lvl, float2 *fpb, const int *__restrict__ fvoff, const float *syn,
                                      const float *wts, float alpha, const float *__restrict__ omega,
                                      const int *__restrict__ vbuf) {
  int c[D];
  {
    int rem = rl;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) { c[d] = rem % g.C[d]; rem /= g.C[d]; }
  }
  int boxbase = 0;
#pragma unroll
  for (int d = D - 1; d >= 0; --d) boxbase += c[d] * g.rst[d];
  if (lane < n) {
    int rem = mem[lane], fo = 0, fs = 1;
#pragma unroll
    for (int d = D - 1; d >= 0; --d) {
      fo += (rem % g.RGP[d] - c[d]) * fs;
      rem /= g.RGP[d];
      fs *= g.FW[d];
    }
    lvl[lane] = fo;
  }
  for (int f = lane; f < g.fp; f += 32) fpb[f] = make_float2(0.f, 0.f);
  __syncwarp();
  add_members_to<PF>(fpb, lvl, fvoff, n, P, MS, lane, syn, wts, alpha, omega, vbuf);
  return boxbase;
}

// ---- mass-conservation sweeps: group tables and the synthesis cache.  Out
// of line: only mass-conserving stages take them, and inlined they cost the
// stage kernels registers. ----

// Group-table entry `slot` (members' region offsets, -1 past the group).
__device__ __noinline__ void export_group(const DJob *sj, int64_t slot, int M, int n, const int *mem, int lane) {
  for (int m = lane; m < M; m += 32) sj->groups[slot * M + m] = m < n ? mem[m] : -1;
  if (lane == 0) sj->gcount[slot] = n;
}

// Members of group-table entry `slot` into mem; returns the group size.
__device__ __noinline__ int table_group_load(const DJob *sj, int64_t slot, int M, int lane, int *mem) {
  const int n = sj->gcount[slot];
  for (int m = lane; m < n; m += 32) mem[m] = sj->groups[slot * M + m];
  __syncwarp();
  return n;
}

// Second sweep from the cache, CQ float4 per lane: the group-table entry
// `slot` (members into mem), the cached synthesis of reference cr (into
// bufA, member rows at vbuf) and its weights, requested together.  Returns
// the group size (0 for a reference without a cache slot).  P is a multiple
// of 4.
template <int CQ>
__device__ __noinline__ int cached_group_load(const DJob *sj, int64_t slot, int64_t cr, int M, int P, int MS,
                                              int lane, int *mem, float *wts, float *bufA,
                                              const int *__restrict__ vbuf) {
  const bool ok = cr < sj->pcache_refs;
  const int gm = lane < M ? sj->groups[slot * M + lane] : 0;
  const int gc = sj->gcount[slot];
  const float wv = (ok && lane < M) ? sj->wcache[cr * M + lane] : 0.f;
  const float4 *pc4 = reinterpret_cast<const float4 *>(sj->pcache + (ok ? cr : 0) * M * P);
  const int nq = ok ? M * P / 4 : 0;
  float4 q[CQ > 0 ? CQ : 1];
#pragma unroll
  for (int k = 0; k < CQ; ++k) {
    const int i = lane + 32 * k;
    q[k] = i < nq ? __ldg(pc4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const int n = ok ? gc : 0;
  if (lane < n) {
    mem[lane] = gm;
    wts[lane] = wv;
  }
#pragma unroll
  for (int k = 0; k < CQ; ++k) {
    const int e = 4 * (lane + 32 * k);
    if (e < n * P) {
      // the four entries belong to one member
      const int m = e / P, v = e - m * P;
      float *d = bufA + m * MS;
      d[vbuf[v]] = q[k].x;
      d[vbuf[v + 1]] = q[k].y;
      d[vbuf[v + 2]] = q[k].z;
      d[vbuf[v + 3]] = q[k].w;
    }
  }
  __syncwarp();
  return n;
}

// The cached synthesis of reference cr (n members of P entries) into bufA
// and its weights into wts.
__device__ __noinline__ void cached_synthesis_load(const DJob *sj, int64_t cr, int M, int n, int P, int MS,
                                                   int lane, float *wts, float *bufA,
                                                   const int *__restrict__ vbuf) {
  const float *pc = sj->pcache + cr * M * P;
  const int tot = n * P;
  for (int e0 = 0; e0 < tot; e0 += 32 * 8) {
    float t[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = e0 + 32 * k + lane;
      t[k] = e < tot ? __ldg(pc + e) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int e = e0 + 32 * k + lane;
      if (e < tot) {
        const int m = e / P, v = e - m * P;
        bufA[m * MS + vbuf[v]] = t[k];
      }
    }
  }
  if (lane < n) wts[lane] = sj->wcache[cr * M + lane];
  __syncwarp();
}

// First sweep: the synthesis (syn, member rows at vbuf) and weights of
// reference cr into the cache.
__device__ __noinline__ void export_synthesis(const DJob *sj, int64_t cr, int M, int n, int P, int MS, int lane,
                                              const float *syn, const float *wts, const int *__restrict__ vbuf) {
  float *pc = sj->pcache + cr * M * P;
  int m = lane / P, v = lane - (lane / P) * P;
  for (int e = lane; e < n * P; e += 32) {
    pc[e] = syn[m * MS + vbuf[v]];
    v += 32;
    while (v >= P) { v -= P; ++m; }
  }
  if (lane < n) sj->wcache[cr * M + lane] = wts[lane];
}

template <int D, int JL, int KB, int MINB, int ST>
__global__ void __launch_bounds__(NW * 32, MINB)
k_stage(const DJob *__restrict__ jobs, int njobs, int total_tiles, int mode, const float *__restrict__ tab,
        int *counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  __shared__ int s_emin;           // lowest set-bit exponent of the staged guide values
  __shared__ unsigned s_vmax;      // largest |value| (float bits)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  DJob *sj = reinterpret_cast<DJob *>(smem);
  int cur_job = -1;
  SmemLayout L;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_tile = atomicAdd(counter, 1);
      s_emin = INT_MAX;
      s_vmax = 0u;
    }
    __syncthreads();
    const int gt = s_tile;
    if (gt >= total_tiles) break;
    int jb;
    {
      int lo = 0, hi = njobs - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
      }
      jb = lo;
    }
    if (jb != cur_job) {
      // new job: its descriptor, per-entry tables and transform matrices
      const int *src = reinterpret_cast<const int *>(&jobs[jb]);
      int *dst = reinterpret_cast<int *>(sj);
      for (int i = threadIdx.x; i < (int)(sizeof(DJob) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      const DGeom &g = sj->g;
      L = smem_layout(smem, g, ST ? ST == 2 : g.stage == 2, mode == 2, mode == 2 && sj->pcache != nullptr);
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
        L.vreg[v] = ro;
        L.vbuf[v] = (v / g.jL) * g.LS + (v % g.jL);
        if (g.kex) {
          int r4 = v, pc = 0;
          for (int d = D - 1; d >= 0; --d) {
            pc |= (r4 % g.j[d]) << (5 * d);
            r4 /= g.j[d];
          }
          L.vcrd[v] = pc;
        }
        if (g.lean) {
          int r3 = v;
          int64_t go = 0;
#pragma unroll
          for (int d = D - 1; d >= 0; --d) {
            go += (int64_t)(r3 % g.j[d]) * g.st[d];
            r3 /= g.j[d];
          }
          L.vgl[v] = go;
        }
        L.omega[v] = w;
        if (v % g.jL == 0) L.rowoff[v / g.jL] = ro;
        if (g.fp) {
          int r2 = v, fo = 0, fs = 1;
#pragma unroll
          for (int d = D - 1; d >= 0; --d) {
            fo += (r2 % g.j[d]) * fs;
            r2 /= g.j[d];
            fs *= g.FW[d];
          }
          L.fvoff[v] = fo;
        }
      }
      for (int f = threadIdx.x; f < g.fp; f += blockDim.x) {
        int r2 = f, ro = 0;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
          ro += (r2 % g.FW[d]) * g.rst[d];
          r2 /= g.FW[d];
        }
        L.fpreg[f] = ro;
      }
      if (threadIdx.x == 0) {
        int o = 0;
        for (int a = 0; a < D; ++a) { L.moff[a] = o; o += mat_block(g.j[a]); }
      }
      {
        int o = 0;
        for (int a = 0; a < D; ++a) {
          const int J = g.j[a];
          // [F | S | F.^2 | F^T]: the DCT with S = F^T, or bior1.5 with its
          // synthesis matrix
          const float *F = tab + (g.spatial ? TAB_BIOR : 0) + gen_off(J);
          const float *S = tab + TAB_BIOR + GEN_TOTAL + gen_off(J);
          for (int e = threadIdx.x; e < J * J; e += blockDim.x) {
            int k = e / J, i = e - k * J;
            const float f = __ldg(F + e), ft = __ldg(F + i * J + k);
            L.mats[o + e] = f;
            L.mats[o + J * J + e] = g.spatial ? __ldg(S + e) : ft;
            L.mats[o + 2 * J * J + e] = f * f;
            L.mats[o + 3 * J * J + e] = ft;
          }
          o += mat_block(J);
        }
      }
      cur_job = jb;
    }
    // sweep 2 only concerns jobs with mass conservation; the others keep the
    // partials of sweep 1, which the second reduce turns into the same output
    if (mode == 2 && sj->groups == nullptr) continue;
    const DGeom &g = sj->g;
    const int tile = gt - sj->tile_base;
    const bool stage2 = ST ? ST == 2 : g.stage == 2;
    const bool mc2 = mode == 2;
    // second sweep from the synthesis cache: y and eta staged, no filtering
    const bool cmode = mc2 && sj->pcache != nullptr;
    const bool leanx = g.lean && !cmode;  // y / eta gathered from global memory
    using SH = CubeShape<D, JL>;
    const int P = SH::fixed ? SH::P : g.P;
    const int MS = SH::fixed ? SH::MS : g.MS;
    // float4 loads per lane of one cached group (compile-time shapes)
    constexpr int CQ = (SH::fixed && SH::P % 4 == 0) ? SH::P * MMAX / 128 : 0;
    const int tile_ref0 = cmode ? sj->ref_base[tile] : 0;
    unsigned char *wp = L.warps + (size_t)warp * L.wbytes;
    int *mem = reinterpret_cast<int *>(wp);
    float *wts = reinterpret_cast<float *>(wp + MMAX * 4);
    float *rr_s = reinterpret_cast<float *>(wp + 2 * MMAX * 4);
    int *lvl = reinterpret_cast<int *>(wp + 3 * MMAX * 4);
    float *bufA = reinterpret_cast<float *>(wp + 4 * MMAX * 4);
    float *bufB = cmode ? bufA : bufA + g.M * MS;
    // the private footprint (float2) follows the group buffer(s), their
    // float count rounded up to even so that it stays 8-byte aligned (one
    // buffer of an odd group size times an odd member stride is odd)
    float2 *fpb = reinterpret_cast<float2 *>(cmode ? bufA + ((g.M * MS + 1) & ~1) : bufB + g.M * MS);
    int64_t *gb = reinterpret_cast<int64_t *>(fpb + g.fp);
    float *Sg = L.Sg, *Sy = L.Sy, *Se = L.Se;
    float2 *acc = L.acc;
    const int *vreg = L.vreg, *vbuf = L.vbuf, *rowoff = L.rowoff;
    const float *omega = L.omega;

    int tc[D], org[D];
    {
      int rem = tile;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) { tc[d] = rem % g.NT[d]; rem /= g.NT[d]; }
#pragma unroll
      for (int d = 0; d < D; ++d) org[d] = tc[d] * g.C[d] - g.rad[d];
    }
    // stage the region(s); locations outside the array are never read as
    // patch entries (candidates are clipped) and are set to zero
    const float *gsrc = sj->guide, *ysrc = sj->y, *esrc = sj->eta;
    const int RS = g.region + RPAD;
    bool nonneg_t = true;
    int emin_t = INT_MAX;
    unsigned vmax_t = 0u;
    // stage-1 Poisson distance: is every staged value s_P times a count
    // K <= PFIX_K / 2 (to a relative 2^-21: float storage and the product
    // with float(1 / s_P) stay below 2^-22)?
    const bool want_counts = !mc2 && !stage2 && g.metric != 0 && g.pfix != nullptr;
    bool counts_t = true;
    for (int e = threadIdx.x; e < RS; e += blockDim.x) {
      float vg = 0.f, vy = 0.f, ve = 0.f;
      if (e < g.region) {
        int rem = e;
        int64_t gi = 0;
        bool in = true;
#pragma unroll
        for (int d = D - 1; d >= 0; --d) {
          int c = rem % g.RGP[d];
          rem /= g.RGP[d];
          int64_t x = (int64_t)org[d] + c;
          if (x < 0 || x >= g.L[d] || c >= g.RG[d]) in = false;  // outside the array, or layout padding
          gi += x * g.st[d];
        }
        if (in) {
          if (cmode) {
            vg = __ldg(ysrc + gi);
            ve = __ldg(esrc + gi);
          } else {
            vg = __ldg(gsrc + gi);
            if (stage2 && !g.lean) vy = __ldg(ysrc + gi);
            if (mc2 && !g.lean) ve = __ldg(esrc + gi);
          }
        }
        acc[e] = make_float2(0.f, 0.f);
      }
      Sg[e] = vg;  // y in the cached sweep
      if (cmode) {
        Se[e] = ve;
      } else {
        if (stage2 && !g.lean) Sy[e] = vy;
        if (mc2 && !g.lean) Se[e] = ve;
      }
      nonneg_t = nonneg_t && vg >= 0.f;
      if (want_counts && vg > 0.f) {
        const float rc = vg * g.inv_sp, kc = rintf(rc);
        counts_t = counts_t && kc <= (float)(PFIX_K / 2) && fabsf(rc - kc) <= 4.76837158e-7f * fmaxf(kc, 1.f);
      }
      if (vg != 0.f) {
        // vg = mant 2^(ex - 150) with a 24-bit mantissa: the exponent of its
        // lowest set bit
        const unsigned bits = __float_as_uint(vg) & 0x7fffffffu;
        const int ex = (int)(bits >> 23);
        const unsigned mant = (bits & 0x7fffffu) | (ex ? 0x800000u : 0u);
        emin_t = min(emin_t, (ex ? ex : 1) - 150 + __ffs(mant) - 1);
        vmax_t = max(vmax_t, bits);
      }
    }
    if (!mc2) {
      if (emin_t != INT_MAX) atomicMin(&s_emin, emin_t);
      if (vmax_t) atomicMax(&s_vmax, vmax_t);
    }
    const bool tile_nonneg = __syncthreads_and(nonneg_t) != 0;
    const bool tile_counts = __syncthreads_and(want_counts && counts_t) != 0;
    // Exact tile (stage-1 SSD, s_P = 2^k, integral gamma): the staged values
    // are multiples of q0 = 2^emin of magnitude at most V q0.  Differences,
    // squares, the SSD, the bias sum, s_P times it and the score are then
    // multiples of u = min(q0^2, q0 s_P) below 2^23 u, all exact in FP32:
    // P (2V)^2 q0^2 for the SSD and gamma 2 P V q0 s_P for gamma B.
    bool tile_exact = false;
    if (g.exact_ok && !mc2 && !stage2) {
      if (s_vmax == 0u) {
        tile_exact = true;
      } else {
        const double q0 = ldexp(1.0, s_emin);
        const double V = (double)__uint_as_float(s_vmax) / q0;
        const double r = g.s_p64 / q0;
        const double unit_rel = r < 1.0 ? r : 1.0;  // u / q0^2
        const double big = (4.0 * g.P * V * V + g.gamma64 * 2.0 * g.P * V * r) / unit_rel;
        tile_exact = big < 8388608.0 && r * 16777216.0 >= 1.0;
      }
    }
    // integer span of the tile's guide values for the exact scores
    int tile_emin = 0, tile_span = 0;
    const float tile_vmax = __uint_as_float(s_vmax);
    if (!mc2 && s_vmax != 0u) {
      tile_emin = s_emin;
      tile_span = (int)(s_vmax >> 23) - 126 - s_emin;  // |v| < 2^(exponent + 1)
    }

    // stage-1 SSD noise bias on a non-negative tile (Prop. "Scaled-Poisson
    // SSD noise bias": B = s_P sum_i (p_i + q_i), every term >= 0): the
    // patch sum of the guide at every region position where a patch fits,
    // so that a candidate's bias is s_P (sum p + sum q) from two reads
    const bool use_bsm = JL > 0 && D <= 2 && g.bsm && !mc2 && !stage2 && g.bias_on && tile_nonneg && g.metric == 0;
    if (use_bsm) {
      // sums along the last axis (into acc[].x, zeroed again below), then
      // along the first; positions whose patch does not fit get 0
      const int RL = g.RGP[D - 1], RLr = g.RG[D - 1], JJL = JL > 0 ? JL : 1;
      float *hs = D == 2 ? reinterpret_cast<float *>(acc) : L.bsm;
      const int hstride = D == 2 ? 2 : 1;
      for (int e = threadIdx.x; e < g.region; e += blockDim.x) {
        float t = 0.f;
        if (e % RL <= RLr - JJL) {
#pragma unroll
          for (int i = 0; i < JJL; ++i) t += Sg[e + i];
        }
        hs[hstride * e] = t;
      }
      if (D == 2) {
        __syncthreads();
        const int R0 = g.RG[0];
        for (int e = threadIdx.x; e < g.region; e += blockDim.x) {
          float t = 0.f;
          if (e / RL <= R0 - JJL) {
#pragma unroll
            for (int r = 0; r < JJL; ++r) t += hs[2 * (e + r * RL)];
          }
          L.bsm[e] = t;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < g.region; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
      }
      __syncthreads();
    }

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
          n = warp_match<D, JL, KB, ST>(g, Sg, rr, org, rowoff, lane, mem, tile_nonneg, tile_exact, tile_emin,
                                        tile_span, tile_vmax, tile_counts, g.diag, use_bsm ? L.bsm : nullptr);
          if (sj->groups) export_group(sj, tslot + ri, g.M, n, mem, lane);
        } else if (CQ > 0 && cmode) {
          // second sweep from the cache: the group-table entry, the cached
          // synthesis and the weights
          n = cached_group_load<CQ>(sj, tslot + ri, (int64_t)tile_ref0 + ri, g.M, P, MS, lane, mem, wts, bufA, vbuf);
        } else {
          n = table_group_load(sj, tslot + ri, g.M, lane, mem);
        }
        if (mode != 1) {
          if (D >= 3 && leanx) {
            // global origin of every member
            if (lane < n) {
              int rem = mem[lane];
              int64_t o = 0;
#pragma unroll
              for (int d = D - 1; d >= 0; --d) {
                o += (int64_t)(org[d] + rem % g.RGP[d]) * g.st[d];
                rem /= g.RGP[d];
              }
              gb[lane] = o;
            }
            __syncwarp();
          }
          // reference slot in the synthesis cache of the first sweep (the
          // cache holds a slot for every possible reference)
          const int64_t cr = sj->pcache ? (int64_t)sj->ref_base[tile] + ri : -1;
          const bool cached = cr >= 0 && cr < sj->pcache_refs;
          if (cmode) {
            // second sweep: the first sweep's synthesis and weights, then
            // only the correction alpha
            if (!cached) n = 0;
            // CQ > 0: loaded with the group
            if (CQ == 0) cached_synthesis_load(sj, cached ? cr : 0, g.M, n, P, MS, lane, wts, bufA, vbuf);
            syn = bufA;
            alpha = mc_alpha<D, SH::P>(g, n, lane, mem, vreg, vbuf, omega, wts, syn, MS, Sg, Se, sj->y, sj->eta,
                                       gb, L.vgl, false);
          } else {
            int which;
            if constexpr (SH::rf)
              which = filter_group_rf<D, JL, ST>(g, n, mc2, lane, mem, vreg, omega, Sg, Sy, Se, bufA, bufB, wts, rr_s,
                                                 sj->y, sj->eta, gb, L.vgl, &alpha, g.diag, L.mats, L.moff, L.vcrd,
                                                 tab);
            else
              which = filter_group<D, JL, ST>(g, n, mc2, lane, mem, vreg, vbuf, omega, Sg, Sy, Se, bufA, bufB, wts,
                                          rr_s, L.mats, L.moff, L.vcrd, tab, sj->y, sj->eta, gb, L.vgl, &alpha,
                                          g.diag);
            syn = which ? bufA : bufB;
            // first sweep of a mass-conserving stage: keep the synthesis
            if (!mc2 && cached && sj->groups) export_synthesis(sj, cr, g.M, n, P, MS, lane, syn, wts, vbuf);
          }
        }
      }
      if (mode == 1) continue;
      // ---- accumulation in the members' order: the warp adds one member
      // after another, lanes over its patch entries (distinct locations), so
      // every location receives its contributions in member order ----
      constexpr int PF = (SH::fixed && SH::P % 32 == 0) ? SH::P : 0;
      int boxbase = 0;
      if (has && g.fp)
        boxbase = fp_export<D, PF>(g, sj->ref_local[tslot + ri], n, P, MS, lane, mem, lvl, fpb, L.fvoff, syn, wts,
                                   alpha, omega, vbuf);
      // ---- ordered, atomic-free accumulation into the tile region ----
      if (!(warp == 0 && rd == 0)) named_sync(1 + warp, 64);
      if (has) {
        if (g.fp) {
          for (int f = lane; f < g.fp; f += 32) {
            float2 t = fpb[f];
            if (t.y != 0.f) {
              int a = boxbase + L.fpreg[f];
              float2 u = acc[a];
              u.x += t.x;
              u.y += t.y;
              acc[a] = u;
            }
          }
        } else {
          add_members_to<PF>(acc, mem, vreg, n, P, MS, lane, syn, wts, alpha, omega, vbuf);
        }
      }
      __threadfence_block();
      {
        int nxt = warp + 1 == NW ? 0 : warp + 1;
        if (!(nxt == 0 && rd == rounds - 1)) named_arrive(1 + nxt, 64);
      }
    }
    if (mode == 1) continue;
    __syncthreads();
    float2 *dst = sj->partial + (int64_t)tile * g.region;
    for (int e = threadIdx.x; e < g.region; e += blockDim.x) dst[e] = acc[e];
  }
}

// Sum the partials of the tiles covering every location in tile order and
// normalize (Def. "Weighted overlap-add estimate").  Locations without weight
// keep the observation.  If write_eta, the denominator is stored as well.
template <int D, int K>
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
    const int64_t u = t - J.vox_base;
    // coordinates (32-bit arithmetic below 2^31 locations)
    int uc[D];
    if (g.N < 2147483648ll) {
      int rem = (int)u;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) {
        const int L = (int)g.L[d];
        uc[d] = rem % L;
        rem /= L;
      }
    } else {
      int64_t rem = u;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) { uc[d] = (int)(rem % g.L[d]); rem /= g.L[d]; }
    }
    // covering tiles per axis: t C - rad <= u <= t C - rad + RG - 1
    int tlo[D], thi[D], tcur[D];
    bool any = true;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int a = uc[d] + g.rad[d] - g.RG[d] + 1;  // t C >= a
      const int b = uc[d] + g.rad[d];                // t C <= b
      int l = a <= 0 ? 0 : (a + g.C[d] - 1) / g.C[d];
      int h = b / g.C[d];
      if (h > g.NT[d] - 1) h = g.NT[d] - 1;
      tlo[d] = l;
      thi[d] = h;
      tcur[d] = l;
      if (l > h) any = false;
    }
    // partials in ascending tile order, K covering tiles per step, all K
    // loads issued before any is added so that their latencies overlap.  The
    // covering tiles are walked by an odometer over their ranges (last axis
    // fastest) that moves a pointer: one step along axis d moves it by
    // step[d] (the next tile's partial, less the core width in the region),
    // a wrap of axis d back by back[d]
    const float2 *__restrict__ p;
    int64_t step[D], back[D];
    {
      int64_t ts = g.region;  // partial-buffer distance of neighbouring tiles along axis d
      int tile = 0;
      int64_t local = 0;
#pragma unroll
      for (int d = D - 1; d >= 0; --d) {
        step[d] = ts - (int64_t)g.C[d] * g.rst[d];
        back[d] = (int64_t)(thi[d] - tlo[d]) * step[d];
        ts *= g.NT[d];
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        tile = tile * g.NT[d] + tcur[d];
        local += (int64_t)(uc[d] + g.rad[d] - tcur[d] * g.C[d]) * g.rst[d];
      }
      p = J.partial + (int64_t)tile * g.region + local;
    }
    float num = 0.f, den = 0.f;
    bool more = any;
    while (more) {
      float2 v[K];
      unsigned valid = 0u;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        v[k] = make_float2(0.f, 0.f);
        if (more) {
          v[k] = *p;
          valid |= 1u << k;
          int d = D - 1;
          while (true) {
            if (++tcur[d] <= thi[d]) {
              p += step[d];
              break;
            }
            tcur[d] = tlo[d];
            p -= back[d];
            if (--d < 0) {
              more = false;
              break;
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if ((valid >> k) & 1u) {
          num += v[k].x;
          den += v[k].y;
        }
      }
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
          int c = rem % g.RGP[d];
          rem /= g.RGP[d];
          lin += ((int64_t)tc[d] * g.C[d] - g.rad[d] + c) * g.st[d];
        }
      }
      groups[slot * g.M + m] = lin;
    }
  }
}

// Exclusive prefix sum of the per-tile reference counts (one CTA of 1024
// threads, contiguous chunks per thread): ref_base[t] = sum_{t' < t} count[t'].
__global__ void __launch_bounds__(1024) k_ref_base(const int *__restrict__ count, int ntiles, int *ref_base) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (ntiles + 1023) / 1024;
  const int lo = min(ntiles, t * per), hi = min(ntiles, lo + per);
  int sum = 0;
  for (int i = lo; i < hi; ++i) sum += count[i];
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int add = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  int run = t ? part[t - 1] : 0;
  for (int i = lo; i < hi; ++i) {
    ref_base[i] = run;
    run += count[i];
  }
}

// ---------------------------------------------------------------------------
// explicit instantiations and launch helpers
// ---------------------------------------------------------------------------

typedef void (*stage_fn)(const DJob *, int, int, int, const float *, int *);

template <int D, int JL, int KB, int ST = 0>
stage_fn stage_ptr(int minb) { return minb >= 2 ? &k_stage<D, JL, KB, 2, ST> : &k_stage<D, JL, KB, 1, ST>; }

// The cubic-patch kernels exist per stage (1 or 2, and 3: stage 1 with a
// Poisson matching distance), which keeps each launch's code to the stage it
// runs -- the SSD kernels carry no Poisson code; all jobs of such a launch
// share it.
template <int D, int JL, int KB>
stage_fn stage_ptr_st(int minb, int stage) {
  return stage == 1 ? stage_ptr<D, JL, KB, 1>(minb)
                    : (stage == 2 ? stage_ptr<D, JL, KB, 2>(minb) : stage_ptr<D, JL, KB, 3>(minb));
}

// Stage kernel for a geometry: D kernel axes, jL > 0 the side of a cubic
// patch (compile-time shape) or 0 for any shape, candidates per lane kb, the
// stage of every job in the launch (1 or 2, 3 for stage 1 with a Poisson
// matching distance; the generic kernels read both from each job), and the
// register budget: minb = 2 limits registers
// so that two CTAs share an SM (used when their shared memory fits), minb = 1
// gives the kernel the whole register file.
stage_fn select_stage_kernel(int D, int jL, int kb, int minb, int stage) {
  switch (D) {
    case 1:
      if (jL == 32 && kb == 5) return stage_ptr_st<1, 32, 5>(minb, stage);
      if (jL == 16 && kb == 4) return stage_ptr_st<1, 16, 4>(minb, stage);
      return stage_ptr<1, 0, 4>(minb);
    case 2:
      if (jL == 8 && kb == 8) return stage_ptr_st<2, 8, 8>(minb, stage);
      if (jL == 4 && kb == 4) return stage_ptr_st<2, 4, 4>(minb, stage);
      return stage_ptr<2, 0, 4>(minb);
    case 3:
      if (jL == 4 && kb == 11) return stage_ptr_st<3, 4, 11>(minb, stage);
      return stage_ptr<3, 0, 4>(minb);
    case 4: return stage_ptr<4, 0, 4>(minb);
    case 5: return stage_ptr<5, 0, 4>(minb);
    case 6: return stage_ptr<6, 0, 4>(minb);
  }
  return nullptr;
}

// FP32 FMA throughput: 8 independent chains per thread, 16 FMAs each per
// iteration (FMA_PEAK_CHAINS per iteration), the result kept alive.
__global__ void __launch_bounds__(256) k_fma_peak(float *out, int iters) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  const float b = 0.9999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

void launch_fma_peak(float *out, int blocks, int threads, int iters) { k_fma_peak<<<blocks, threads>>>(out, iters); }

void launch_ref_base(const int *count, int ntiles, int *ref_base, cudaStream_t st) {
  k_ref_base<<<1, 1024, 0, st>>>(count, ntiles, ref_base);
}

void launch_reduce(int D, const DJob *jobs, int njobs, int64_t total, int write_eta, int grid,
                   cudaStream_t st) {
  switch (D) {
    case 1: k_reduce<1, 8><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 2: k_reduce<2, 8><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 3: k_reduce<3, 8><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 4: k_reduce<4, 8><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 5: k_reduce<5, 8><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
    case 6: k_reduce<6, 8><<<grid, 256, 0, st>>>(jobs, njobs, total, write_eta); break;
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

void launch_sched_mark(const SGeom &s, unsigned char *flags, cudaStream_t st) {
  int64_t total = s.nslots * s.passes;
  int grid = (int)((total + 255) / 256);
  if (grid > 148 * 16) grid = 148 * 16;
  if (grid < 1) grid = 1;
  k_sched_mark<<<grid, 256, 0, st>>>(s, flags);
}

void launch_coverage(const CovGeom &c, const unsigned char *flags, int32_t *cov, unsigned long long *sums,
                     cudaStream_t st) {
  const int64_t total = c.N > c.nflags ? c.N : c.nflags;
  int grid = (int)((total + 255) / 256);
  if (grid > 148 * 16) grid = 148 * 16;
  if (grid < 1) grid = 1;
  k_coverage<<<grid, 256, 0, st>>>(c, flags, cov, sums);
}

cudaError_t set_stage_smem(stage_fn f, int bytes) {
  return cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace bmnd
