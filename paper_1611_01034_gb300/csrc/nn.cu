// Learned gauge-covariant preconditioner layer (an addition to the method:
// the paper has no learned parts).  Two linear parallel-transport
// convolutions N = L2 o L1 (1 -> 8 -> 1 spinor channels):
//
//     y_o(x) = sum_i sum_d W[o][i][d] (T_d psi_i)(x),   d = self, +-T, +-Z, +-Y, +-X,
//     (T_{+mu} psi)(x) = U_mu(x) psi(x + mu),  (T_{-mu} psi)(x) = U_mu(x - mu)^dagger psi(x - mu),
//
// W[o][i][d] a complex 4 x 4 spin matrix acting trivially on colour, the
// fermion boundary factor on hops across T.  The preconditioner applies
// z = B(v) + N(v - D B(v)).  Kernels: the layer (one thread per site and
// output channel, FP32 arithmetic, hidden channels stored in FP32 or FP16),
// the same kernel with conjugate-transposed, direction-reversed weights as the
// adjoint layer, and the weight gradient sum_x g_o(x) (T_d psi_i)(x)^dagger
// (per-CTA partial sums over a tile of sites, reduced in FP64 in a second pass).
#include <cuda_fp16.h>

#include "tm_kernels.h"

namespace tmamg {

namespace {

constexpr int kNdir = 9;

// fine field in the library's chunked layout: rhs r, channel c at f + (r * C + c) * 24 V
struct FineIn {
  const float* f;
  int C;
  __device__ __forceinline__ void load(long V, int r, int c, long s, cx<float> (&p)[12]) const {
    ld_cx<float, 12>(f + ((long)r * C + c) * NR_SPINOR * V, V, s, p);
  }
};
struct FineOut {
  float* f;
  int C;
  __device__ __forceinline__ void store(long V, int r, int c, long s, const cx<float> (&p)[12], bool acc) const {
    float* base = f + ((long)r * C + c) * NR_SPINOR * V;
    if (acc) {
      cx<float> q[12];
      ld_cx<float, 12>(base, V, s, q);
#pragma unroll
      for (int k = 0; k < 12; ++k) q[k] = q[k] + p[k];
      st_cx<float, 12>(base, V, s, q);
    } else {
      st_cx<float, 12>(base, V, s, p);
    }
  }
};
// hidden channels: [rhs][C][V][12 complex] contiguous per site, FP32 or FP16
template <typename Th>
struct HiddenIn {
  const Th* f;
  int C;
  __device__ __forceinline__ void load(long V, int r, int c, long s, cx<float> (&p)[12]) const {
    const Th* q = f + (((long)r * C + c) * V + s) * 24;
    if constexpr (sizeof(Th) == 4) {
      const float4* v = reinterpret_cast<const float4*>(q);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const float4 a = v[k];
        p[2 * k] = cx<float>{a.x, a.y};
        p[2 * k + 1] = cx<float>{a.z, a.w};
      }
    } else {
      const __half2* v = reinterpret_cast<const __half2*>(q);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float2 a = __half22float2(v[k]);
        p[k] = cx<float>{a.x, a.y};
      }
    }
  }
};
template <typename Th>
struct HiddenOut {
  Th* f;
  int C;
  __device__ __forceinline__ void store(long V, int r, int c, long s, const cx<float> (&p)[12], bool) const {
    Th* q = f + (((long)r * C + c) * V + s) * 24;
    if constexpr (sizeof(Th) == 4) {
      float4* v = reinterpret_cast<float4*>(q);
#pragma unroll
      for (int k = 0; k < 6; ++k) v[k] = make_float4(p[2 * k].r, p[2 * k].i, p[2 * k + 1].r, p[2 * k + 1].i);
    } else {
      __half2* v = reinterpret_cast<__half2*>(q);
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = __floats2half2_rn(p[k].r, p[k].i);
    }
  }
};

// phi = T_d psi_c(x) at site s (coordinates cs) of rhs r
template <class In>
__device__ __forceinline__ void transported(const In& in, const float* __restrict__ gauge, const Lat& g, float bc,
                                            int r, int ch, int s, const int (&cs)[4], int d, cx<float> (&phi)[12]) {
  if (d == 0) {
    in.load(g.V, r, ch, s, phi);
    return;
  }
  const int mu = (d - 1) >> 1;
  const bool fwd = ((d - 1) & 1) == 0;
  const int nb = fwd ? nb_fwd(g, s, cs, mu) : nb_bwd(g, s, cs, mu);
  const float sg = (mu == 0 && (fwd ? cs[0] == g.L[0] - 1 : cs[0] == 0)) ? bc : 1.f;
  cx<float> p[12];
  in.load(g.V, r, ch, nb, p);
  Link<float> U;
  ld_link(gauge, g.V, mu, fwd ? s : nb, U);
#pragma unroll
  for (int sp = 0; sp < 4; ++sp) {
    cx<float> x[3] = {sg * p[3 * sp], sg * p[3 * sp + 1], sg * p[3 * sp + 2]}, y[3];
    if (fwd)
      su3_mul(U, x, y);
    else
      su3_dag_mul(U, x, y);
    phi[3 * sp] = y[0];
    phi[3 * sp + 1] = y[1];
    phi[3 * sp + 2] = y[2];
  }
}

// one layer: thread per (site, output channel); blockIdx.y = rhs
template <class In, class Out, int CIN, int COUT>
__global__ void __launch_bounds__(128) k_layer(In in, Out out, const float* __restrict__ gauge,
                                               const float2* __restrict__ W, Lat g, float bc, int accumulate) {
  __shared__ float2 Ws[COUT * CIN * kNdir * 16];
  for (int e = threadIdx.x; e < COUT * CIN * kNdir * 16; e += blockDim.x) Ws[e] = W[e];
  __syncthreads();
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)g.V * COUT) return;
  const int o = (int)(idx / g.V), s = (int)(idx % g.V), r = blockIdx.y;
  int cs[4];
  site_coords(g, s, cs);
  cx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cx<float>{0.f, 0.f};
  for (int d = 0; d < kNdir; ++d)
    for (int i = 0; i < CIN; ++i) {
      cx<float> phi[12];
      transported(in, gauge, g, bc, r, i, s, cs, d, phi);
      const float2* w = Ws + ((o * CIN + i) * kNdir + d) * 16;
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const cx<float> wst{w[sp * 4 + t].x, w[sp * 4 + t].y};
#pragma unroll
          for (int c = 0; c < 3; ++c) cfma(acc[3 * sp + c], wst, phi[3 * t + c]);
        }
    }
  out.store(g.V, r, o, s, acc, accumulate != 0);
}

template <class In, class Out, int CIN, int COUT>
void run_layer(In in, Out out, const float* gauge, const float2* W, const Lat& g, double bc, int nrhs, bool acc,
               cudaStream_t st) {
  const long tot = (long)g.V * COUT;
  dim3 grid((unsigned)((tot + 127) / 128), nrhs);
  k_layer<In, Out, CIN, COUT><<<grid, 128, 0, st>>>(in, out, gauge, W, g, (float)bc, acc ? 1 : 0);
}

// weight gradient partials: CTA = 64 sites of one rhs; partial[cta][o][i][d][s][t] =
// sum over its sites and colours of g_o(x)[s] conj(phi_{i,d}(x)[t])
constexpr int kGradSites = 64;
template <class In, class G, int CIN, int COUT>
__global__ void __launch_bounds__(128) k_wgrad(In in, G gin, const float* __restrict__ gauge, Lat g, float bc,
                                               float2* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<float>* gs = reinterpret_cast<cx<float>*>(smem_raw);  // [COUT][64][12]
  cx<float>* ph = gs + COUT * kGradSites * 12;              // [64][12]
  cx<float>* red = ph + kGradSites * 12;                    // [128]
  constexpr int E = COUT * 16;
  constexpr int NG = 128 / E;
  const int r = blockIdx.y;
  const long s0 = (long)blockIdx.x * kGradSites;
  const int tid = threadIdx.x;
  for (int e = tid; e < COUT * kGradSites; e += blockDim.x) {
    const int o = e / kGradSites, k = e % kGradSites;
    cx<float> p[12];
    if (s0 + k < g.V) {
      gin.load(g.V, r, o, s0 + k, p);
    } else {
#pragma unroll
      for (int q = 0; q < 12; ++q) p[q] = cx<float>{0.f, 0.f};
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) gs[(o * kGradSites + k) * 12 + q] = p[q];
  }
  const long cta = (long)blockIdx.y * gridDim.x + blockIdx.x;
  const int grp = tid / E, ent = tid % E;
  const int o = ent / 16, sp = (ent % 16) / 4, t = ent % 4;
  for (int i = 0; i < CIN; ++i)
    for (int d = 0; d < kNdir; ++d) {
      __syncthreads();
      if (tid < kGradSites) {
        cx<float> phi[12];
        const long s = s0 + tid;
        if (s < g.V) {
          int cs[4];
          site_coords(g, (int)s, cs);
          transported(in, gauge, g, bc, r, i, (int)s, cs, d, phi);
        } else {
#pragma unroll
          for (int q = 0; q < 12; ++q) phi[q] = cx<float>{0.f, 0.f};
        }
#pragma unroll
        for (int q = 0; q < 12; ++q) ph[tid * 12 + q] = phi[q];
      }
      __syncthreads();
      cx<float> sum{0.f, 0.f};
      if (grp < NG)
        for (int k = grp; k < kGradSites; k += NG)
#pragma unroll
          for (int c = 0; c < 3; ++c) cfmac(sum, ph[k * 12 + 3 * t + c], gs[(o * kGradSites + k) * 12 + 3 * sp + c]);
      red[tid] = sum;
      __syncthreads();
      if (tid < E) {
        cx<float> tot = red[tid];
        for (int q = 1; q < NG; ++q) tot = tot + red[q * E + tid];
        const long nct = (long)gridDim.x * gridDim.y;
        partial[(((long)o * CIN + i) * kNdir * 16 + d * 16 + sp * 4 + t) * nct + cta] = make_float2(tot.r, tot.i);
      }
    }
}

// out[e] = sum_cta partial[cta][e] in FP64
__global__ void k_wgrad_reduce(const float2* __restrict__ partial, long ncta, double2* __restrict__ out) {
  __shared__ double red[2 * 128];
  const int e = blockIdx.x;
  double a = 0, b = 0;
  for (long c = threadIdx.x; c < ncta; c += blockDim.x) {
    const float2 v = partial[(long)e * ncta + c];
    a += v.x;
    b += v.y;
  }
  red[threadIdx.x] = a;
  red[128 + threadIdx.x] = b;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[threadIdx.x] += red[threadIdx.x + w];
      red[128 + threadIdx.x] += red[128 + threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = make_double2(red[0], red[128]);
}

template <class In, class G, int CIN, int COUT>
void run_wgrad(In in, G gin, const float* gauge, const Lat& g, double bc, int nrhs, float2* partial, double2* out,
               cudaStream_t st) {
  const int nx = (g.V + kGradSites - 1) / kGradSites;
  const size_t smem = (size_t)(COUT * kGradSites * 12 + kGradSites * 12 + 128) * sizeof(cx<float>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_wgrad<In, G, CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  dim3 grid(nx, nrhs);
  k_wgrad<In, G, CIN, COUT><<<grid, 128, smem, st>>>(in, gin, gauge, g, (float)bc, partial);
  const int nent = COUT * CIN * kNdir * 16;
  k_wgrad_reduce<<<nent, 128, 0, st>>>(partial, (long)nx * nrhs, out);
}

}  // namespace

long nn_wgrad_partial_floats2(const Lat& g, int nrhs) {
  return (long)((g.V + kGradSites - 1) / kGradSites) * nrhs * kNnHidden * kNdir * 16;
}

void nn_layer1(const float* r, void* hid, bool half, const float* gauge, const float2* W1, const Lat& g, double bc,
               int nrhs, cudaStream_t st) {
  if (half)
    run_layer<FineIn, HiddenOut<__half>, 1, kNnHidden>(FineIn{r, 1}, HiddenOut<__half>{static_cast<__half*>(hid),
                                                                                         kNnHidden},
                                                      gauge, W1, g, bc, nrhs, false, st);
  else
    run_layer<FineIn, HiddenOut<float>, 1, kNnHidden>(FineIn{r, 1}, HiddenOut<float>{static_cast<float*>(hid),
                                                                                       kNnHidden},
                                                     gauge, W1, g, bc, nrhs, false, st);
}

void nn_layer2(const void* hid, bool half, float* y, bool accumulate, const float* gauge, const float2* W2,
               const Lat& g, double bc, int nrhs, cudaStream_t st) {
  if (half)
    run_layer<HiddenIn<__half>, FineOut, kNnHidden, 1>(HiddenIn<__half>{static_cast<const __half*>(hid), kNnHidden},
                                                      FineOut{y, 1}, gauge, W2, g, bc, nrhs, accumulate, st);
  else
    run_layer<HiddenIn<float>, FineOut, kNnHidden, 1>(HiddenIn<float>{static_cast<const float*>(hid), kNnHidden},
                                                     FineOut{y, 1}, gauge, W2, g, bc, nrhs, accumulate, st);
}

void nn_layer2_adjoint(const float* gy, float* gh, const float* gauge, const float2* W2adj, const Lat& g, double bc,
                       int nrhs, cudaStream_t st) {
  run_layer<FineIn, HiddenOut<float>, 1, kNnHidden>(FineIn{gy, 1}, HiddenOut<float>{gh, kNnHidden}, gauge, W2adj, g,
                                                   bc, nrhs, false, st);
}

void nn_grad_w2(const float* hid, const float* gy, const float* gauge, const Lat& g, double bc, int nrhs,
                float2* partial, double2* out, cudaStream_t st) {
  run_wgrad<HiddenIn<float>, FineIn, kNnHidden, 1>(HiddenIn<float>{hid, kNnHidden}, FineIn{gy, 1}, gauge, g, bc,
                                                  nrhs, partial, out, st);
}

void nn_grad_w1(const float* r, const float* gh, const float* gauge, const Lat& g, double bc, int nrhs,
                float2* partial, double2* out, cudaStream_t st) {
  run_wgrad<FineIn, HiddenIn<float>, 1, kNnHidden>(FineIn{r, 1}, HiddenIn<float>{gh, kNnHidden}, gauge, g, bc, nrhs,
                                                  partial, out, st);
}

}  // namespace tmamg
