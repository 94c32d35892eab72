// Coarse odd-even stencil on the 5th-generation tensor cores (tcgen05, TF32
// inputs, FP32 accumulation in tensor memory).
//
// The batched odd-even Schur complement of the coarse operator (Sec. 3: the
// coarsest level is solved by odd-even preconditioned GMRES; Sec. 1: D_c is a
// 9-point stencil of 2N_v x 2N_v blocks) is, per target site k and for R
// right-hand sides at once,
//
//     y(k) = sum_t A_t(k) x_t(nbr(k, t)),
//
// a sum of dense complex (n x n) x (n x R) products, n = 2 N_v.  Each product
// is one tcgen05.mma chain: the operator block is the A operand (M = 2n real
// rows: row 2i holds Re A[i][.], row 2i+1 holds Im A[i][.]; padded to 128),
// the gathered source vectors are the B operand (N = 2 R_pad columns: Re of
// every rhs, then Im of every rhs), and TMEM accumulates
//     D = [[Re A Re x, Re A Im x]; [Im A Re x, Im A Im x]]
// interleaved by rows, so Re y = D[2i][q] - D[2i+1][R_pad+q] and
// Im y = D[2i][R_pad+q] + D[2i+1][q] combine two neighbouring TMEM lanes of
// the same warp (one shuffle).
//
// Operator blocks are kept pre-tiled in HBM in the K-major UMMA layout with
// 64-byte swizzle (the layout the tensor core reads without shared-memory bank
// conflicts), so one bulk TMA copy (cp.async.bulk) moves a whole block into
// shared memory.  Targets:
//   odd  sites: u_o = sum_{t=1..8} [D_oo^-1 B_t] v_e(nb_t)   (blocks premultiplied)
//   even sites: y_e = A_self v_e - sum_{t=1..8} B_t u_o(nb_t) + i mu_c Gamma5_c v_e
// TF32 keeps 10 explicit mantissa bits; `split` adds the residual parts
// (x - tf32(x), and for split 3 also A - tf32(A) read from a second tile set)
// as extra products so the sum reaches FP32-level accuracy (3xTF32).
//
// Warp roles in a persistent CTA (one per SM): warp 0 issues the bulk copies
// of the operator tiles, warp 1 owns TMEM and issues the MMAs, warps 2-3
// gather and convert the source vectors into the B operand, warps 4-7 read
// the accumulators and write y.  Every mbarrier wait is bounded; on a timeout
// the CTA records ERRF_TIMEOUT, drains its copies and MMAs (bounded) and
// releases TMEM.
#include <cstdint>

#include "tm_kernels.h"

namespace tmamg {

namespace {

constexpr int kGatherWarps = 8;                            // warps 2 .. 9
constexpr int kIssuers = 2;                                // MMA issuing warps 1 and 14
constexpr int kTcThreads = (2 + kGatherWarps + 4 + 1) * 32;  // + epilogue warps 10 .. 13, issuer 14
constexpr uint32_t kSpinLimit = 1u << 22;
// independent accumulators per target: consecutive MMAs rotate over them so the
// tensor pipe never waits for the previous product into the same TMEM columns
constexpr int kAcc = 4;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on phase `parity` (at most `limit` polls); false on timeout or
// when another warp aborted
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort,
                                          uint32_t limit = kSpinLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (mbar_test(b, parity)) return true;
    if ((it & 255u) == 255u && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 64-byte swizzle (8-row atoms of
// 64-byte rows, 512 bytes apart), start address advanced within an atom row
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  return (uint64_t)((su32(p) >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(512u >> 4) << 32) | (1ull << 46) |
         (4ull << 61);
}

// instruction descriptor: kind::tf32, D F32, A/B TF32, both K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_tf32(int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* out) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of FP32 element (row, k) in a K-major tile with 64-byte swizzle:
// K is cut into chunks of 16 elements (64 bytes), each chunk holds all `rows`
// rows at 64 bytes apiece, and inside every 512-byte block the 16-byte unit
// index is XORed with (row / 2) mod 4.  Chunks are 512-byte aligned when rows
// is a multiple of 8.
__host__ __device__ __forceinline__ uint32_t tile_off(int row, int k, int rows) {
  const uint32_t o = (uint32_t)row * 64u + (uint32_t)(k & 15) * 4u;
  return (uint32_t)(k >> 4) * (uint32_t)rows * 64u + (o ^ (((o >> 7) & 3u) << 4));
}

struct TcArgs {
  const float* tiles;     // [ntgt][nt] tiles of mp x kp floats
  const float* tiles_lo;  // split 3: A - tf32(A), same layout
  const int* nbr;         // [ntgt][nt] source index (compact)
  const float* src0;      // source of t = 0 (null: t = 0 reads src1 like the others)
  const float* src1;
  float sign1;            // factor on src1 values
  long s0_str, s1_str;    // per-rhs strides (floats)
  float* out;
  long o_str;
  const float* diag;      // out += i mu Gamma5_c diag(k) (null: none)
  long d_str;
  float mu;
  const int* active;      // rhs mask (null: all)
  int ntgt, nt, n, nv, kp, mp, R, rp, split, stages;
  int* err;
  uint32_t spin;          // polls per pipeline wait before giving up (the drain waits use kSpinLimit)
};

struct TcShared {
  uint64_t full_a[16], full_b[16], empty[16], tfull[2], tempty[2], drain;
  uint32_t tmem_base;
  int abort;
};

__global__ void __launch_bounds__(kTcThreads, 1) k_tc_stencil(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  __shared__ TcShared sh;
  // swizzle atoms need 512-byte alignment of every tile: align the base explicitly
  unsigned char* smem = smem_dyn + ((1024u - (su32(smem_dyn) & 1023u)) & 1023u);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.stages, N = 2 * a.rp;
  const uint32_t TB = (uint32_t)a.mp * a.kp * 4;  // operator tile bytes
  const uint32_t BB = (uint32_t)N * a.kp * 4;     // B operand bytes
  const uint32_t guard = (uint32_t)(128 - a.mp) * 64u;  // rows mp..127 of the last chunk
  unsigned char* A = smem;
  unsigned char* Alo = A + (size_t)S * TB;
  unsigned char* Bh = Alo + (a.split == 3 ? (size_t)S * TB : 0) + guard;
  unsigned char* Bl = Bh + (size_t)S * BB;
  const int ncol_need = 2 * kAcc * N;  // two target slots of kAcc accumulators
  const uint32_t ncols = ncol_need <= 32 ? 32 : (ncol_need <= 64 ? 64 : (ncol_need <= 128 ? 128 : (ncol_need <= 256 ? 256 : 512)));
  volatile int* abort = &sh.abort;

  // zero the B operands once: padded rows (rhs >= R) and columns (k >= n) stay zero
  {
    const size_t words = (size_t)S * BB / 4 * (a.split >= 2 ? 2 : 1);
    uint32_t* z = reinterpret_cast<uint32_t*>(Bh);
    for (size_t i = threadIdx.x; i < words; i += blockDim.x) z[i] = 0u;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&sh.full_a[s], 1);
      mbar_init(&sh.full_b[s], 1);
      mbar_init(&sh.empty[s], kIssuers);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sh.tfull[i], kIssuers);
      mbar_init(&sh.tempty[i], 4);
    }
    mbar_init(&sh.drain, kIssuers);
    sh.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before();
  __syncthreads();
  tc_after();
  const uint32_t tmem = sh.tmem_base;
  auto fail = [&]() {
    sh.abort = 1;
    atomicOr(a.err, ERRF_TIMEOUT);
  };

  if (warp == 0) {
    // ---- operator tiles: bulk copies -------------------------------------------
    if (lane == 0) {
      long g = 0;
      bool ok = true;
      for (int k = blockIdx.x; k < a.ntgt && ok; k += gridDim.x)
        for (int t = 0; t < a.nt && ok; ++t, ++g) {
          const int s = (int)(g % S);
          if (!mbar_wait(&sh.empty[s], (uint32_t)((g / S) & 1) ^ 1u, abort, a.spin)) {
            ok = false;
            break;
          }
          const size_t off = ((size_t)k * a.nt + t) * (TB / 4);
          mbar_expect_tx(&sh.full_a[s], a.split == 3 ? 2 * TB : TB);
          bulk_g2s(A + (size_t)s * TB, a.tiles + off, TB, &sh.full_a[s]);
          if (a.split == 3) bulk_g2s(Alo + (size_t)s * TB, a.tiles_lo + off, TB, &sh.full_a[s]);
        }
      if (!ok) {
        fail();
        // drain: every copy issued lands before the CTA leaves (bounded waits)
        const long g0 = g > S ? g - S : 0;
        for (long q = g0; q < g; ++q) {
          volatile int never = 0;
          mbar_wait(&sh.full_a[q % S], (uint32_t)((q / S) & 1), &never);
        }
      }
    }
  } else if (warp == 1 || warp == 2 + kGatherWarps + 4) {
    // ---- MMA issue: two issuing threads, MMA ci of a target goes to issuer ci % 2 and
    // accumulator ci % kAcc (a single issuing thread cannot keep the tensor pipe busy
    // with these small products) -------------------------------------------------------------
    const int iss = warp == 1 ? 0 : 1;
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(N);
      long g = 0;
      int j = 0;
      bool ok = true;
      for (int k = blockIdx.x; k < a.ntgt && ok; k += gridDim.x, ++j) {
        const int slot = j & 1;
        if (!mbar_wait(&sh.tempty[slot], (uint32_t)((j >> 1) & 1) ^ 1u, abort, a.spin)) {
          ok = false;
          break;
        }
        tc_after();
        const uint32_t d0 = tmem + (uint32_t)(slot * kAcc * N);
        int ci = 0;  // MMA counter within the target: accumulator ci % kAcc, overwrite on first use
        for (int t = 0; t < a.nt; ++t, ++g) {
          const int s = (int)(g % S);
          const uint32_t par = (uint32_t)((g / S) & 1);
          if (!mbar_wait(&sh.full_b[s], par, abort, a.spin)) {  // the gather warp saw the tile land
            ok = false;
            break;
          }
          tc_after();
          const unsigned char* As = A + (size_t)s * TB;
          const unsigned char* Als = Alo + (size_t)s * TB;
          const unsigned char* Bs = Bh + (size_t)s * BB;
          const unsigned char* Bls = Bl + (size_t)s * BB;
          for (int ks = 0; ks < a.kp / 8; ++ks) {
            const uint32_t ao = (uint32_t)(ks >> 1) * (uint32_t)a.mp * 64u + (uint32_t)(ks & 1) * 32u;
            const uint32_t bo = (uint32_t)(ks >> 1) * (uint32_t)N * 64u + (uint32_t)(ks & 1) * 32u;
            const uint64_t ad = sdesc(As + ao);
            const uint64_t bd = sdesc(Bs + bo);
            if (ci % kIssuers == iss) mma_tf32(d0 + (uint32_t)((ci % kAcc) * N), ad, bd, idesc, ci >= kAcc ? 1u : 0u);
            ++ci;
            if (a.split >= 2) {
              if (ci % kIssuers == iss)
                mma_tf32(d0 + (uint32_t)((ci % kAcc) * N), ad, sdesc(Bls + bo), idesc, ci >= kAcc ? 1u : 0u);
              ++ci;
            }
            if (a.split == 3) {
              if (ci % kIssuers == iss)
                mma_tf32(d0 + (uint32_t)((ci % kAcc) * N), sdesc(Als + ao), bd, idesc, ci >= kAcc ? 1u : 0u);
              ++ci;
            }
          }
          mma_commit(&sh.empty[s]);
        }
        if (!ok) break;
        mma_commit(&sh.tfull[slot]);
      }
      if (!ok) fail();
      // every MMA issued has completed before TMEM is released
      mma_commit(&sh.drain);
      volatile int never = 0;
      if (!mbar_wait(&sh.drain, 0u, &never)) atomicOr(a.err, ERRF_TIMEOUT);
    }
  } else if (warp < 2 + kGatherWarps) {
    // ---- B operand: gather, sign, split, store ------------------------------------------
    // gather warp w fills stages w, w + G, ...; lane = (rhs q mod 8) * 4 + (k mod 4), so a
    // warp's stores cover one 128-byte row group of a core-matrix column (no bank conflicts).
    // G <= S keeps every waiter within one phase of its stage's empty barrier (the parity
    // test cannot tell phases two apart).
    const int w = warp - 2;
    const int G = kGatherWarps < S ? kGatherWarps : S;
    const int qq = lane >> 2, cc = lane & 3;
    const int nq = a.rp >> 3, nc4 = (a.n + 3) >> 2;
    int ntl = 0;
    for (int k = blockIdx.x; k < a.ntgt; k += gridDim.x) ++ntl;
    const long total = (long)ntl * a.nt;
    bool ok = true;
    for (long g = w; w < G && g < total; g += G) {
      const int jl = (int)(g / a.nt), t = (int)(g % a.nt);
      const int k = blockIdx.x + jl * gridDim.x;
      const int j = a.nbr[(long)k * a.nt + t];
      const int s = (int)(g % S);
      if (!mbar_wait(&sh.empty[s], (uint32_t)((g / S) & 1) ^ 1u, abort, a.spin)) {
        ok = false;
        break;
      }
      const bool self = t == 0 && a.src0;
      const float* src = self ? a.src0 : a.src1;
      const long str = self ? a.s0_str : a.s1_str;
      const float sg = self ? 1.f : a.sign1;
      unsigned char* Bs = Bh + (size_t)s * BB;
      unsigned char* Bls = Bl + (size_t)s * BB;
      constexpr int U = 4;
      for (int p0 = 0; p0 < nq * nc4; p0 += U) {
        float2 v[U];
        int qv[U], cv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int pr = p0 + u;
          qv[u] = (pr / nc4) * 8 + qq;
          cv[u] = (pr % nc4) * 4 + cc;
          v[u] = make_float2(0.f, 0.f);
          if (pr < nq * nc4 && qv[u] < a.R && cv[u] < a.n && (!a.active || a.active[qv[u]]))
            v[u] = reinterpret_cast<const float2*>(src + qv[u] * str)[(long)j * a.n + cv[u]];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (p0 + u >= nq * nc4 || qv[u] >= a.R || cv[u] >= a.n) continue;
          const float re = sg * v[u].x, im = sg * v[u].y;
          const float rh = tf32_round(re), ih = tf32_round(im);
          *reinterpret_cast<float*>(Bs + tile_off(qv[u], cv[u], N)) = rh;
          *reinterpret_cast<float*>(Bs + tile_off(a.rp + qv[u], cv[u], N)) = ih;
          if (a.split >= 2) {
            *reinterpret_cast<float*>(Bls + tile_off(qv[u], cv[u], N)) = re - rh;
            *reinterpret_cast<float*>(Bls + tile_off(a.rp + qv[u], cv[u], N)) = im - ih;
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        // the stage is ready once its operator tile has landed as well
        if (!mbar_wait(&sh.full_a[s], (uint32_t)((g / S) & 1), abort, a.spin)) ok = false;
        else mbar_arrive(&sh.full_b[s]);
      }
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
    }
    if (!ok && lane == 0) fail();
  } else {
    // ---- epilogue: TMEM -> registers -> y ---------------------------------------------------
    const int q4 = warp & 3;
    const int m = q4 * 32 + lane;  // TMEM lane = real row 2i + p
    const int row = m >> 1, p = m & 1;
    const bool live = m < 2 * a.n;
    float acc[64];
    int j = 0;
    bool ok = true;
    for (int k = blockIdx.x; k < a.ntgt; k += gridDim.x, ++j) {
      const int slot = j & 1;
      if (!mbar_wait(&sh.tfull[slot], (uint32_t)((j >> 1) & 1), abort, a.spin)) {
        ok = false;
        break;
      }
      tc_after();
      const uint32_t base = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(slot * kAcc * N);
      for (int c0 = 0; c0 < N; c0 += 16) tmem_ld16(base + (uint32_t)c0, acc + c0);
      for (int ai = 1; ai < kAcc; ++ai)
        for (int c0 = 0; c0 < N; c0 += 16) {
          float part[16];
          tmem_ld16(base + (uint32_t)(ai * N + c0), part);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[c0 + i] += part[i];
        }
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.tempty[slot]);
      for (int q = 0; q < a.R; ++q) {
        const float x = __shfl_xor_sync(0xffffffffu, acc[a.rp + q], 1);
        float val = p == 0 ? acc[q] - x : acc[q] + x;
        if (live && (!a.active || a.active[q])) {
          if (a.diag) {
            const float* dv = a.diag + q * a.d_str + (long)k * 2 * a.n + 2 * row;
            const float g5 = row < a.nv ? -a.mu : a.mu;
            val += p == 0 ? -g5 * dv[1] : g5 * dv[0];
          }
          a.out[q * a.o_str + (long)k * 2 * a.n + m] = val;
        }
      }
    }
    if (!ok && lane == 0) fail();
  }
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------
// tile builders (CUDA cores; once per coarse build or mu change)
// ---------------------------------------------------------------------------
// even targets: tile t = B_t(site) for t = 0..8 (block 0 = self, mu-free)
__global__ void k_tc_tiles_even(const float* __restrict__ Dc, float* __restrict__ tiles, float* __restrict__ lo,
                                OEGeom oe, int kp, int mp) {
  const int k = blockIdx.x, t = blockIdx.y, n = 2 * oe.nv;
  const int site = oe.even_site[k];
  const cx<float>* B = reinterpret_cast<const cx<float>*>(Dc) + ((long)site * 9 + t) * n * n;
  float* out = tiles + ((long)k * 9 + t) * mp * kp;
  float* outl = lo ? lo + ((long)k * 9 + t) * mp * kp : nullptr;
  for (int e = threadIdx.x; e < mp * kp; e += blockDim.x) {
    const int c = e / mp, mm = e % mp;
    float v = 0.f;
    if (mm < 2 * n && c < n) {
      const cx<float> b = B[(long)c * n + (mm >> 1)];
      v = (mm & 1) ? b.i : b.r;
    }
    const float h = tf32_round(v);
    out[tile_off(mm, c, mp) / 4] = h;
    if (outl) outl[tile_off(mm, c, mp) / 4] = v - h;
  }
}

// odd targets: tile t - 1 = D_oo^-1(k) B_t(site) for t = 1..8
__global__ void k_tc_tiles_odd(const float* __restrict__ Dc, const float* __restrict__ Dinv,
                               float* __restrict__ tiles, float* __restrict__ lo, OEGeom oe, int kp, int mp) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int k = blockIdx.x, t = blockIdx.y + 1, n = 2 * oe.nv;
  cx<float>* Ds = reinterpret_cast<cx<float>*>(sm_raw);  // [col][row]
  cx<float>* Bs = Ds + n * n;
  const int site = oe.odd_site[k];
  const cx<float>* Di = reinterpret_cast<const cx<float>*>(Dinv) + (long)k * n * n;
  const cx<float>* B = reinterpret_cast<const cx<float>*>(Dc) + ((long)site * 9 + t) * n * n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    Ds[e] = Di[e];
    Bs[e] = B[e];
  }
  __syncthreads();
  float* out = tiles + ((long)k * 8 + t - 1) * mp * kp;
  float* outl = lo ? lo + ((long)k * 8 + t - 1) * mp * kp : nullptr;
  for (int e = threadIdx.x; e < mp * kp; e += blockDim.x) {
    const int c = e / mp, mm = e % mp;
    float v = 0.f;
    if (mm < 2 * n && c < n) {
      const int r = mm >> 1;
      cx<float> acc{0.f, 0.f};
      for (int l = 0; l < n; ++l) cfma(acc, Ds[(long)l * n + r], Bs[(long)c * n + l]);
      v = (mm & 1) ? acc.i : acc.r;
    }
    const float h = tf32_round(v);
    out[tile_off(mm, c, mp) / 4] = h;
    if (outl) outl[tile_off(mm, c, mp) / 4] = v - h;
  }
}

// site reached by stencil block t (0 self, 1 + 2 mu forward, 2 + 2 mu backward)
__device__ __forceinline__ int tc_nb(const Lat& g, int s, int t) {
  if (t == 0) return s;
  int c[4];
  site_coords(g, s, c);
  const int mu = (t - 1) >> 1;
  return ((t - 1) & 1) ? nb_bwd(g, s, c, mu) : nb_fwd(g, s, c, mu);
}

// neighbour tables: even targets [nhalf][9] (self, then odd compact index of
// each hop), odd targets [nhalf][8] (even compact index of each hop)
__global__ void k_tc_nbr(OEGeom oe, int* nbr_e, int* nbr_o) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= oe.nhalf) return;
  const int se = oe.even_site[k], so = oe.odd_site[k];
  nbr_e[k * 9] = k;
  for (int t = 1; t < 9; ++t) {
    nbr_e[k * 9 + t] = oe.cidx[tc_nb(oe.gc, se, t)];
    nbr_o[k * 8 + t - 1] = oe.cidx[tc_nb(oe.gc, so, t)];
  }
}

int g_sms = 0;

int tc_stages(const TcGeom& tg, int R, int split) {
  const int rp = (R + 7) / 8 * 8, N = 2 * rp;
  const long TB = (long)tg.mp * tg.kp * 4, BB = (long)N * tg.kp * 4;
  const long guard = (128L - tg.mp) * 64;
  const long per = TB * (split == 3 ? 2 : 1) + BB * (split >= 2 ? 2 : 1);
  long s = (kTcSmemBytes - 1024 - guard) / per;
  return (int)(s > 16 ? 16 : s);
}

void launch_tc(const TcArgs& a, cudaStream_t st) {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_tc_stencil, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
  }
  const int grid = a.ntgt < g_sms ? a.ntgt : g_sms;
  k_tc_stencil<<<grid, kTcThreads, kTcSmemBytes, st>>>(a);
}

}  // namespace

bool tc_supported(int nv, int nrhs, int split) {
  if (2 * nv > 64 || nrhs < 1 || nrhs > 32 || split < 1 || split > 3) return false;
  TcGeom tg{};
  tg.kp = (2 * nv + 15) / 16 * 16;
  tg.mp = (4 * nv + 7) / 8 * 8;
  return tc_stages(tg, nrhs, split) >= 2;
}

void tc_build(const float* Dc, const float* Dinv, const OEGeom& oe, const TcGeom& tg, cudaStream_t st) {
  k_tc_nbr<<<(oe.nhalf + 127) / 128, 128, 0, st>>>(oe, tg.nbr_e, tg.nbr_o);
  dim3 ge(oe.nhalf, 9);
  k_tc_tiles_even<<<ge, 256, 0, st>>>(Dc, tg.even, tg.even_lo, oe, tg.kp, tg.mp);
  tc_build_odd(Dc, Dinv, oe, tg, st);
}

void tc_build_odd(const float* Dc, const float* Dinv, const OEGeom& oe, const TcGeom& tg, cudaStream_t st) {
  const int n = 2 * oe.nv;
  const size_t smem = (size_t)2 * n * n * sizeof(cx<float>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_tiles_odd, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr = true;
  }
  dim3 go(oe.nhalf, 8);
  k_tc_tiles_odd<<<go, 256, smem, st>>>(Dc, Dinv, tg.odd, tg.odd_lo, oe, tg.kp, tg.mp);
}

void launch_tc_schur(const TcGeom& tg, const OEGeom& oe, const float* ve, float* uo, float* ye, double mu_c,
                     int nrhs, long vstr, long ustr, long ystr, const int* active, int split, int* err,
                     cudaStream_t st, unsigned spin) {
  TcArgs a{};
  a.spin = spin ? spin : kSpinLimit;
  a.n = 2 * oe.nv;
  a.nv = oe.nv;
  a.kp = tg.kp;
  a.mp = tg.mp;
  a.R = nrhs;
  a.rp = (nrhs + 7) / 8 * 8;
  a.split = split;
  a.stages = tc_stages(tg, nrhs, split);
  a.active = active;
  a.err = err;
  a.ntgt = oe.nhalf;
  // u_o = sum_t [D_oo^-1 B_t] v_e(nb_t)
  a.tiles = tg.odd;
  a.tiles_lo = tg.odd_lo;
  a.nbr = tg.nbr_o;
  a.nt = 8;
  a.src0 = nullptr;
  a.src1 = ve;
  a.s1_str = vstr;
  a.sign1 = 1.f;
  a.out = uo;
  a.o_str = ustr;
  a.diag = nullptr;
  launch_tc(a, st);
  // y_e = A_self v_e - sum_t B_t u_o(nb_t) + i mu_c Gamma5_c v_e
  a.tiles = tg.even;
  a.tiles_lo = tg.even_lo;
  a.nbr = tg.nbr_e;
  a.nt = 9;
  a.src0 = ve;
  a.s0_str = vstr;
  a.src1 = uo;
  a.s1_str = ustr;
  a.sign1 = -1.f;
  a.out = ye;
  a.o_str = ystr;
  a.diag = ve;
  a.d_str = vstr;
  a.mu = (float)mu_c;
  launch_tc(a, st);
}

}  // namespace tmamg
