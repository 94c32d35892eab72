// Internal device/host helpers shared by the CUDA translation units of the
// twisted-mass DD-alphaAMG library.  Nothing here is part of the C ABI.
//
// Field layout ("chunked SoA"): a site field with NR reals per site is stored
// as [NR / 4][V] chunks of 4 reals (two complex numbers): one float4 in FP32,
// two consecutive double2 in FP64.  One warp's load of one chunk is 512 (FP32)
// or 1024 (FP64) contiguous bytes, and both precisions share one index map
// (real r of site s at ((r / 4) * V + s) * 4 + r % 4), so precision casts and
// mixed-precision vector operations can run on the flat arrays.  A spinor has 24 reals
// (12 complex, index 3*spin + colour), a link 12 reals (rows 0 and 1 of the
// SU(3) matrix; row 2 is rebuilt as conj(row0 x row1)), a clover site 72
// reals (two Hermitian 6x6 chiral blocks, 36 reals each: 6 real diagonal
// entries then the 15 upper-triangle entries (0,1),(0,2),...,(4,5)).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace tmamg {

// ---------------------------------------------------------------------------
// complex arithmetic
// ---------------------------------------------------------------------------
template <typename T>
struct cx {
  T r, i;
};

template <typename T>
__host__ __device__ __forceinline__ cx<T> mkc(T r, T i) { return cx<T>{r, i}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a) { return {-a.r, -a.i}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.r, s * a.i}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.r, -a.i}; }
// conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r};
}
// acc += a * b
template <typename T>
__host__ __device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.r = fma(a.r, b.r, acc.r);
  acc.r = fma(-a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i);
  acc.i = fma(a.i, b.r, acc.i);
}
// acc += conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ void cfmac(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.r = fma(a.r, b.r, acc.r);
  acc.r = fma(a.i, b.i, acc.r);
  acc.i = fma(a.r, b.i, acc.i);
  acc.i = fma(-a.i, b.r, acc.i);
}
template <typename T>
__host__ __device__ __forceinline__ T norm2(cx<T> a) { return a.r * a.r + a.i * a.i; }

// multiply by a phase from {+1, +i, -1, -i}, coded 0, 1, 2, 3
template <int P, typename T>
__device__ __forceinline__ cx<T> mulph(cx<T> z) {
  if constexpr (P == 0) return z;
  else if constexpr (P == 1) return {-z.i, z.r};
  else if constexpr (P == 2) return {-z.r, -z.i};
  else return {z.i, -z.r};
}
__host__ __device__ constexpr int conjph(int p) { return (4 - p) & 3; }

// ---------------------------------------------------------------------------
// gamma matrices in the chiral basis
//   gamma_mu = [[0, A_mu], [A_mu^dagger, 0]], gamma5 = diag(-1, -1, +1, +1)
// lattice direction mu = 0..3 is T, Z, Y, X and carries gamma_4, gamma_3,
// gamma_2, gamma_1:  A_T = -1, A_Z = -i sigma_3, A_Y = -i sigma_2,
// A_X = -i sigma_1.  Every A_mu is monomial: row r has the single entry
// phase[r] in column perm[r].
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int gperm(int mu, int r) {
  return (mu < 2) ? r : 1 - r;
}
__host__ __device__ constexpr int gphase(int mu, int r) {
  // T: {-1,-1}; Z: {-i,+i}; Y: {-1,+1}; X: {-i,-i}
  return mu == 0 ? 2 : mu == 1 ? (r == 0 ? 3 : 1) : mu == 2 ? (r == 0 ? 2 : 0) : 3;
}

// ---------------------------------------------------------------------------
// lattice geometry (T, Z, Y, X; X fastest)
// ---------------------------------------------------------------------------
struct Lat {
  int L[4];
  int V;
  int st[4];  // site-index stride of each direction
};

inline Lat make_lat(const int L[4]) {
  Lat g;
  for (int d = 0; d < 4; ++d) g.L[d] = L[d];
  g.st[3] = 1;
  g.st[2] = L[3];
  g.st[1] = L[3] * L[2];
  g.st[0] = L[3] * L[2] * L[1];
  g.V = L[0] * L[1] * L[2] * L[3];
  return g;
}

__host__ __device__ __forceinline__ void site_coords(const Lat& g, int s, int c[4]) {
  c[3] = s % g.L[3];
  int q = s / g.L[3];
  c[2] = q % g.L[2];
  q /= g.L[2];
  c[1] = q % g.L[1];
  c[0] = q / g.L[1];
}

__host__ __device__ __forceinline__ int nb_fwd(const Lat& g, int s, const int c[4], int mu) {
  return c[mu] + 1 < g.L[mu] ? s + g.st[mu] : s - (g.L[mu] - 1) * g.st[mu];
}
__host__ __device__ __forceinline__ int nb_bwd(const Lat& g, int s, const int c[4], int mu) {
  return c[mu] > 0 ? s - g.st[mu] : s + (g.L[mu] - 1) * g.st[mu];
}

// ---------------------------------------------------------------------------
// chunked SoA loads and stores
// ---------------------------------------------------------------------------
// load NC complex numbers of site s from a chunked field with V sites
template <typename T, int NC>
__device__ __forceinline__ void ld_cx(const T* __restrict__ base, long V, long s, cx<T> (&z)[NC]) {
  static_assert(NC % 2 == 0, "chunks hold two complex numbers");
  if constexpr (sizeof(T) == 8) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) {
      const double2* q = p + 2 * (k * V + s);
      double2 v0 = __ldg(q), v1 = __ldg(q + 1);
      z[2 * k] = cx<T>{(T)v0.x, (T)v0.y};
      z[2 * k + 1] = cx<T>{(T)v1.x, (T)v1.y};
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) {
      float4 v = __ldg(p + k * V + s);
      z[2 * k] = cx<T>{(T)v.x, (T)v.y};
      z[2 * k + 1] = cx<T>{(T)v.z, (T)v.w};
    }
  }
}

template <typename T, int NC>
__device__ __forceinline__ void st_cx(T* __restrict__ base, long V, long s, const cx<T> (&z)[NC]) {
  static_assert(NC % 2 == 0, "chunks hold two complex numbers");
  if constexpr (sizeof(T) == 8) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) {
      double2* q = p + 2 * (k * V + s);
      q[0] = make_double2((double)z[2 * k].r, (double)z[2 * k].i);
      q[1] = make_double2((double)z[2 * k + 1].r, (double)z[2 * k + 1].i);
    }
  } else {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < NC / 2; ++k)
      p[k * V + s] = make_float4((float)z[2 * k].r, (float)z[2 * k].i, (float)z[2 * k + 1].r,
                                 (float)z[2 * k + 1].i);
  }
}

// ---------------------------------------------------------------------------
// 16-bit storage of operators read by the FP32 K-cycle (values of TM_F16 /
// TM_BF16); a complex number is one 32-bit word (re, im), a chunk of two
// complex numbers 8 bytes, so a 16-bit copy keeps the element order of the
// FP32 array it was made from
// ---------------------------------------------------------------------------
constexpr int ST_NATIVE = 0, ST_F16 = 2, ST_BF16 = 3;

template <int S>
__device__ __forceinline__ float2 unpack16x2(unsigned u) {
  if constexpr (S == ST_F16) {
    __half2 v;
    memcpy(&v, &u, 4);
    return __half22float2(v);
  } else {
    __nv_bfloat162 v;
    memcpy(&v, &u, 4);
    return __bfloat1622float2(v);
  }
}

// NC complex numbers of site s from a chunked field stored in 16 bits
template <typename T, int S, int NC>
__device__ __forceinline__ void ld_cx16(const void* __restrict__ base, long V, long s, cx<T> (&z)[NC]) {
  static_assert(NC % 2 == 0, "chunks hold two complex numbers");
  const uint2* p = reinterpret_cast<const uint2*>(base);
#pragma unroll
  for (int k = 0; k < NC / 2; ++k) {
    const uint2 v = __ldg(p + k * V + s);
    const float2 a = unpack16x2<S>(v.x), b = unpack16x2<S>(v.y);
    z[2 * k] = cx<T>{(T)a.x, (T)a.y};
    z[2 * k + 1] = cx<T>{(T)b.x, (T)b.y};
  }
}

// load NR reals of site s (NR a multiple of 4)
template <typename T, int NR>
__device__ __forceinline__ void ld_re(const T* __restrict__ base, long V, long s, T (&r)[NR]) {
  if constexpr (sizeof(T) == 8) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < NR / 4; ++k) {
      const double2* q = p + 2 * (k * V + s);
      double2 v0 = __ldg(q), v1 = __ldg(q + 1);
      r[4 * k] = v0.x;
      r[4 * k + 1] = v0.y;
      r[4 * k + 2] = v1.x;
      r[4 * k + 3] = v1.y;
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < NR / 4; ++k) {
      float4 v = __ldg(p + k * V + s);
      r[4 * k] = v.x;
      r[4 * k + 1] = v.y;
      r[4 * k + 2] = v.z;
      r[4 * k + 3] = v.w;
    }
  }
}

template <typename T, int NR>
__device__ __forceinline__ void st_re(T* __restrict__ base, long V, long s, const T (&r)[NR]) {
  if constexpr (sizeof(T) == 8) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < NR / 4; ++k) {
      double2* q = p + 2 * (k * V + s);
      q[0] = make_double2(r[4 * k], r[4 * k + 1]);
      q[1] = make_double2(r[4 * k + 2], r[4 * k + 3]);
    }
  } else {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < NR / 4; ++k)
      p[k * V + s] = make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
  }
}

// reals per site of the packed fields
constexpr int NR_SPINOR = 24;
constexpr int NR_LINK = 12;
constexpr int NR_CLOVER = 72;

// ---------------------------------------------------------------------------
// SU(3) link: rows 0, 1 stored; row 2 = conj(row0 x row1)
// ---------------------------------------------------------------------------
template <typename T>
struct Link {
  cx<T> u[3][3];
};

template <typename T>
__device__ __forceinline__ void link_from_rows(const cx<T> (&z)[6], Link<T>& U) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    U.u[0][k] = z[k];
    U.u[1][k] = z[3 + k];
  }
  U.u[2][0] = conj(U.u[0][1] * U.u[1][2] - U.u[0][2] * U.u[1][1]);
  U.u[2][1] = conj(U.u[0][2] * U.u[1][0] - U.u[0][0] * U.u[1][2]);
  U.u[2][2] = conj(U.u[0][0] * U.u[1][1] - U.u[0][1] * U.u[1][0]);
}

template <typename T>
__device__ __forceinline__ void ld_link(const T* __restrict__ gauge, long V, int mu, long s, Link<T>& U) {
  cx<T> z[6];
  ld_cx<T, 6>(gauge + (long)mu * NR_LINK * V, V, s, z);
  link_from_rows(z, U);
}

// the link from links stored as T (S = ST_NATIVE) or in 16 bits (ST_F16, ST_BF16)
template <typename T, int S>
__device__ __forceinline__ void ld_link_s(const void* __restrict__ gauge, long V, int mu, long s, Link<T>& U) {
  if constexpr (S == ST_NATIVE) {
    ld_link(static_cast<const T*>(gauge), V, mu, s, U);
  } else {
    cx<T> z[6];
    ld_cx16<T, S, 6>(static_cast<const unsigned short*>(gauge) + (long)mu * NR_LINK * V, V, s, z);
    link_from_rows(z, U);
  }
}

// NR reals of site s, stored as T or in 16 bits (chunks of 4 reals)
template <typename T, int S, int NR>
__device__ __forceinline__ void ld_re_s(const void* __restrict__ base, long V, long s, T (&r)[NR]) {
  if constexpr (S == ST_NATIVE) {
    ld_re<T, NR>(static_cast<const T*>(base), V, s, r);
  } else {
    const uint2* p = reinterpret_cast<const uint2*>(base);
#pragma unroll
    for (int k = 0; k < NR / 4; ++k) {
      const uint2 v = __ldg(p + k * V + s);
      const float2 a = unpack16x2<S>(v.x), b = unpack16x2<S>(v.y);
      r[4 * k] = (T)a.x;
      r[4 * k + 1] = (T)a.y;
      r[4 * k + 2] = (T)b.x;
      r[4 * k + 3] = (T)b.y;
    }
  }
}

// NC complex numbers of site s, stored as T or in 16 bits
template <typename T, int S, int NC>
__device__ __forceinline__ void ld_cx_s(const void* __restrict__ base, long V, long s, cx<T> (&z)[NC]) {
  if constexpr (S == ST_NATIVE)
    ld_cx<T, NC>(static_cast<const T*>(base), V, s, z);
  else
    ld_cx16<T, S, NC>(base, V, s, z);
}

// y = U x (colour)
template <typename T>
__device__ __forceinline__ void su3_mul(const Link<T>& U, const cx<T> (&x)[3], cx<T> (&y)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<T> acc = U.u[a][0] * x[0];
    cfma(acc, U.u[a][1], x[1]);
    cfma(acc, U.u[a][2], x[2]);
    y[a] = acc;
  }
}
// y = U^dagger x
template <typename T>
__device__ __forceinline__ void su3_dag_mul(const Link<T>& U, const cx<T> (&x)[3], cx<T> (&y)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cx<T> acc = cmulc(U.u[0][a], x[0]);
    cfmac(acc, U.u[1][a], x[1]);
    cfmac(acc, U.u[2][a], x[2]);
    y[a] = acc;
  }
}

// ---------------------------------------------------------------------------
// clover block apply: y6 = M x6, M Hermitian 6x6 packed as 36 reals
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void herm6_mul(const T* m, const cx<T>* x, cx<T>* y) {
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i] = m[i] * x[i];
  int k = 6;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      cx<T> u{m[k], m[k + 1]};
      k += 2;
      cfma(y[i], u, x[j]);
      cfmac(y[j], u, x[i]);
    }
  }
}

// ---------------------------------------------------------------------------
// error flags set by kernels (bitwise OR into a device int)
// ---------------------------------------------------------------------------
enum : int {
  ERRF_NOT_SU3 = 1,
  ERRF_RANK = 2,
  ERRF_SINGULAR = 4,
  ERRF_NONFINITE = 8,
  ERRF_TIMEOUT = 16,  // a bounded device-side wait ran out
};

// ---------------------------------------------------------------------------
// block reduction helpers (blockDim.x a multiple of 32, <= 1024)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reduce N values across the block; on return every thread holds the sums.
// smem must hold 32 * N values of T.
template <typename T, int N>
__device__ __forceinline__ void block_allreduce(T (&v)[N], T* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) smem[warp * N + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T s = 0;
    for (int w = 0; w < nw; ++w) s += smem[w * N + k];
    v[k] = s;
  }
}

// sum over the CTA of 16 values per thread; thread t < 16 gets sum t in fin[t].
// Inside a warp a reduce-scatter (16 + 8 + 4 + 2 + 1 + 1 shuffles instead of
// 16 x 5) leaves lane L with the warp sum of value 8 b4 + 4 b3 + 2 b2 + b1
// (b_k bit k of L); the warps' sums are then added by 16 threads.
template <typename T>
__device__ __forceinline__ void block_reduce16(const T (&d)[16], T* red, T* fin) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T v8[8], v4[4], v2[2];
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int m = 0; m < 8; ++m) v8[m] = (hi ? d[8 + m] : d[m]) + __shfl_xor_sync(full, hi ? d[m] : d[8 + m], 16);
  }
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int m = 0; m < 4; ++m) v4[m] = (hi ? v8[4 + m] : v8[m]) + __shfl_xor_sync(full, hi ? v8[m] : v8[4 + m], 8);
  }
  {
    const bool hi = lane & 4;
#pragma unroll
    for (int m = 0; m < 2; ++m) v2[m] = (hi ? v4[2 + m] : v4[m]) + __shfl_xor_sync(full, hi ? v4[m] : v4[2 + m], 4);
  }
  const bool hi = lane & 2;
  T v1 = (hi ? v2[1] : v2[0]) + __shfl_xor_sync(full, hi ? v2[0] : v2[1], 2);
  v1 += __shfl_xor_sync(full, v1, 1);
  if (!(lane & 1)) red[warp * 16 + ((lane >> 1) & 15)] = v1;
  __syncthreads();
  if (threadIdx.x < 16) {
    T sum = 0;
    for (int w = 0; w < nw; ++w) sum += red[w * 16 + threadIdx.x];
    fin[threadIdx.x] = sum;
  }
  __syncthreads();
}

}  // namespace tmamg
