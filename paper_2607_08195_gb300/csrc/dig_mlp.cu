// dig_mlp.cu -- learned per-cell closure: MLP 13 -> 64 -> 64 -> 64 -> 8 with
// GELU, BF16 weights and activations, FP32 accumulation on the tensor cores.
// Inference (S12: the coupling's closure and closure_forward) runs on the
// fifth-generation tensor cores: tcgen05.mma with FP32 accumulators in
// tensor memory, 128 rows per tile (k_mlp_forward_tc).  Training (S13):
// forward and backward of 64 rows per CTA with WMMA m16n16k16 tiles, weight
// gradients dW = delta^T A over the rows accumulated into FP32; Adam on the
// FP32 master parameters.
//
// Parameter layout (FP32 master, [out][in] per layer): W1[64][13] b1[64]
// W2[64][64] b2[64] W3[64][64] b3[64] W4[8][64] b4[8].  In shared memory the
// weights are BF16 [out][in] with the input dimension of layer 1 padded to 16
// and the outputs of layer 4 padded to 16 (zeros).
#include "dig_internal.h"

#include <cuda_bf16.h>
#include <mma.h>

namespace dig {

namespace {
using namespace nvcuda;
constexpr int NIN = 13, NH = 64, NOUT = 8, PIN = 16, POUT = 16;
constexpr int ROWS = 64;       // rows per CTA
constexpr int MT = 128;        // threads per CTA (4 warps)
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH, OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + NOUT * NH,
              NPARAM = OFF_B4 + NOUT;
static_assert(NPARAM == 9736, "parameter count");

struct Smem {
  __nv_bfloat16 W1[NH * PIN], W2[NH * NH], W3[NH * NH], W4[POUT * NH];
  float b1[NH], b2[NH], b3[NH], b4[POUT];
  __nv_bfloat16 X[ROWS * PIN];
  __nv_bfloat16 A1[ROWS * NH], A2[ROWS * NH], A3[ROWS * NH];
  float G1[ROWS * NH], G2[ROWS * NH], G3[ROWS * NH];  // GELU'(z) per layer
  float Y[ROWS * POUT];
  float F[ROWS * NH];                                 // FP32 GEMM staging
  __nv_bfloat16 D[ROWS * NH];                         // BF16 delta of the current layer
  __nv_bfloat16 D4[ROWS * POUT];
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678f)) + z * expf(-0.5f * z * z) * 0.39894228f;
}

__device__ void load_params(Smem& S, const float* __restrict__ p) {
  for (int i = threadIdx.x; i < NH * PIN; i += MT) {
    const int j = i / PIN, k = i % PIN;
    S.W1[i] = __float2bfloat16_rn(k < NIN ? p[OFF_W1 + j * NIN + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH * NH; i += MT) {
    S.W2[i] = __float2bfloat16_rn(p[OFF_W2 + i]);
    S.W3[i] = __float2bfloat16_rn(p[OFF_W3 + i]);
  }
  for (int i = threadIdx.x; i < POUT * NH; i += MT) {
    const int j = i / NH;
    S.W4[i] = __float2bfloat16_rn(j < NOUT ? p[OFF_W4 + i] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH; i += MT) {
    S.b1[i] = p[OFF_B1 + i];
    S.b2[i] = p[OFF_B2 + i];
    S.b3[i] = p[OFF_B3 + i];
  }
  for (int i = threadIdx.x; i < POUT; i += MT) S.b4[i] = i < NOUT ? p[OFF_B4 + i] : 0.0f;
}

// out[ROWS x N] (FP32, ld N) = A[ROWS x K] (bf16 row-major, ld K) * W^T, W = [N][K] row-major
template <int K, int N>
__device__ void gemm_AWt(const __nv_bfloat16* A, const __nv_bfloat16* W, float* out) {
  const int warp = threadIdx.x >> 5;
  constexpr int TM = ROWS / 16, TN = N / 16;
  for (int t = warp; t < TM * TN; t += MT / 32) {
    const int tm = t / TN, tn = t % TN;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
    wmma::fill_fragment(acc, 0.0f);
#pragma unroll
    for (int k = 0; k < K; k += 16) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> a;
      wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::col_major> b;
      wmma::load_matrix_sync(a, A + tm * 16 * K + k, K);
      wmma::load_matrix_sync(b, W + tn * 16 * K + k, K);
      wmma::mma_sync(acc, a, b, acc);
    }
    wmma::store_matrix_sync(out + tm * 16 * N + tn * 16, acc, N, wmma::mem_row_major);
  }
}

// out[ROWS x N] = D[ROWS x K] (bf16 row-major, ld K) * W, W = [K][N] row-major
template <int K, int N>
__device__ void gemm_DW(const __nv_bfloat16* Dm, const __nv_bfloat16* W, float* out) {
  const int warp = threadIdx.x >> 5;
  constexpr int TM = ROWS / 16, TN = N / 16;
  for (int t = warp; t < TM * TN; t += MT / 32) {
    const int tm = t / TN, tn = t % TN;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
    wmma::fill_fragment(acc, 0.0f);
#pragma unroll
    for (int k = 0; k < K; k += 16) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> a;
      wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
      wmma::load_matrix_sync(a, Dm + tm * 16 * K + k, K);
      wmma::load_matrix_sync(b, W + k * N + tn * 16, N);
      wmma::mma_sync(acc, a, b, acc);
    }
    wmma::store_matrix_sync(out + tm * 16 * N + tn * 16, acc, N, wmma::mem_row_major);
  }
}

// out[M x N] = D^T A over the ROWS rows: D [ROWS x M] (ld M), A [ROWS x N] (ld N)
template <int M, int N>
__device__ void gemm_DtA(const __nv_bfloat16* Dm, const __nv_bfloat16* A, float* out) {
  const int warp = threadIdx.x >> 5;
  constexpr int TM = M / 16, TN = N / 16;
  for (int t = warp; t < TM * TN; t += MT / 32) {
    const int tm = t / TN, tn = t % TN;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
    wmma::fill_fragment(acc, 0.0f);
#pragma unroll
    for (int r = 0; r < ROWS; r += 16) {
      wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::col_major> a;
      wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> b;
      wmma::load_matrix_sync(a, Dm + r * M + tm * 16, M);
      wmma::load_matrix_sync(b, A + r * N + tn * 16, N);
      wmma::mma_sync(acc, a, b, acc);
    }
    wmma::store_matrix_sync(out + tm * 16 * N + tn * 16, acc, N, wmma::mem_row_major);
  }
}

// forward of the CTA's rows; keeps the BF16 activations and GELU'(z)
__device__ void forward(Smem& S, const float* __restrict__ X, long long row0, long long n) {
  for (int i = threadIdx.x; i < ROWS * PIN; i += MT) {
    const int r = i / PIN, k = i % PIN;
    const long long g = row0 + r;
    S.X[i] = __float2bfloat16_rn(g < n && k < NIN ? X[g * NIN + k] : 0.0f);
  }
  __syncthreads();
  gemm_AWt<PIN, NH>(S.X, S.W1, S.F);
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
    const float z = S.F[i] + S.b1[i % NH];
    S.A1[i] = __float2bfloat16_rn(gelu(z));
    S.G1[i] = gelu_d(z);
  }
  __syncthreads();
  gemm_AWt<NH, NH>(S.A1, S.W2, S.F);
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
    const float z = S.F[i] + S.b2[i % NH];
    S.A2[i] = __float2bfloat16_rn(gelu(z));
    S.G2[i] = gelu_d(z);
  }
  __syncthreads();
  gemm_AWt<NH, NH>(S.A2, S.W3, S.F);
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
    const float z = S.F[i] + S.b3[i % NH];
    S.A3[i] = __float2bfloat16_rn(gelu(z));
    S.G3[i] = gelu_d(z);
  }
  __syncthreads();
  gemm_AWt<NH, POUT>(S.A3, S.W4, S.Y);
  __syncthreads();
  for (int i = threadIdx.x; i < ROWS * POUT; i += MT) S.Y[i] += S.b4[i % POUT];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Inference on tcgen05.  One CTA of 128 threads loops over tiles of 128 rows.
// Per layer one thread issues the MMAs (K = 16 per instruction) into an FP32
// accumulator of 128 TMEM lanes x N columns and commits them to an mbarrier;
// after the wait every warp reads its 32 lanes (tcgen05.ld 32x32b), adds the
// bias, applies GELU and rounds to BF16 into the next layer's operand in
// shared memory.  Operands are in the canonical no-swizzle K-major layout:
// core matrices of 8 rows x 8 BF16 (16 bytes a row, 128 contiguous bytes),
// core matrices adjacent along K 128 bytes apart (leading byte offset),
// 8-row groups K/8 x 128 bytes apart (stride byte offset).  A: the tile's
// rows [128 x K]; B: the weights [N x K] ([out][in], K-major), so D = A W^T.
// Layers 1-3 accumulate into TMEM columns 0..63 (N = 64), layer 4 into
// columns 64..79 (N = 16: the 8 outputs and 8 zero rows of padding).
// Every wait on the mbarrier gives up after about a second: the CTA then
// records the failure in *status, frees its TMEM and returns.  With hold != 0
// (a test of that path) no MMA is issued or committed, so the first wait
// runs out.
// ---------------------------------------------------------------------------
constexpr int TROWS = 128;          // rows per tile (MMA M)
constexpr int TCT = 128;            // threads per CTA
constexpr uint32_t TMEM_COLS = 128; // allocated TMEM columns (64 + 16 used)

struct TcSmem {
  alignas(128) __nv_bfloat16 W1[NH * PIN];
  alignas(128) __nv_bfloat16 W2[NH * NH];
  alignas(128) __nv_bfloat16 W3[NH * NH];
  alignas(128) __nv_bfloat16 W4[POUT * NH];
  alignas(128) __nv_bfloat16 X[TROWS * PIN];
  alignas(128) __nv_bfloat16 H[TROWS * NH];
  float b1[NH], b2[NH], b3[NH], b4[POUT];
  alignas(8) unsigned long long mbar;
  uint32_t tmem;
};
// four CTAs per SM at most (the dynamic allocation below is padded to a
// quarter of the SM's shared memory), so that their TMEM (4 x 128 columns)
// fits the SM's 512 columns and no allocation has to wait
constexpr size_t TC_SMEM = 56 * 1024;
static_assert(sizeof(TcSmem) <= TC_SMEM, "tcgen05 MLP shared memory");

// element offset of (row r, column k) of an operand with K columns
__device__ __forceinline__ int cofs(int r, int k, int K) {
  return (r >> 3) * (K * 8) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

// shared-memory matrix descriptor: start address, leading byte offset 128,
// stride byte offset K x 16 bytes (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mdesc(const void* base, int K) {
  const uint32_t a = smem_u32(base);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(((uint32_t)K * 16u) & 0x3FFFFu) >> 4 << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the completion of phase `parity` of the mbarrier, at most ~1 s
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// bias, GELU and BF16 of the thread's row (TMEM lane = row) into S.H
__device__ __forceinline__ void tc_hidden(TcSmem& S, uint32_t tl, const float* b) {
  const int row = threadIdx.x;
#pragma unroll
  for (int c = 0; c < NH; c += 16) {
    uint32_t r[16];
    tmem_ld16(tl + (uint32_t)c, r);
    tmem_wait_ld();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      uint32_t pk[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = c + 8 * h + 2 * e;
        pk[e] = pack_bf16(gelu(__uint_as_float(r[8 * h + 2 * e]) + b[j]),
                          gelu(__uint_as_float(r[8 * h + 2 * e + 1]) + b[j + 1]));
      }
      *reinterpret_cast<uint4*>(S.H + cofs(row, c + 8 * h, NH)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
}

__global__ void __launch_bounds__(TCT) k_mlp_forward_tc(const float* __restrict__ p, const float* __restrict__ X,
                                                       long long n, float* __restrict__ Y, int* __restrict__ status,
                                                       int hold) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  // weights (BF16, canonical layout) and biases
  for (int i = tid; i < NH * PIN; i += TCT) {
    const int j = i / PIN, k = i % PIN;
    S.W1[cofs(j, k, PIN)] = __float2bfloat16_rn(k < NIN ? p[OFF_W1 + j * NIN + k] : 0.0f);
  }
  for (int i = tid; i < NH * NH; i += TCT) {
    const int j = i / NH, k = i % NH;
    S.W2[cofs(j, k, NH)] = __float2bfloat16_rn(p[OFF_W2 + i]);
    S.W3[cofs(j, k, NH)] = __float2bfloat16_rn(p[OFF_W3 + i]);
  }
  for (int i = tid; i < POUT * NH; i += TCT) {
    const int j = i / NH, k = i % NH;
    S.W4[cofs(j, k, NH)] = __float2bfloat16_rn(j < NOUT ? p[OFF_W4 + i] : 0.0f);
  }
  for (int i = tid; i < NH; i += TCT) {
    S.b1[i] = p[OFF_B1 + i];
    S.b2[i] = p[OFF_B2 + i];
    S.b3[i] = p[OFF_B3 + i];
  }
  if (tid < POUT) S.b4[tid] = tid < NOUT ? p[OFF_B4 + tid] : 0.0f;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's 32 lanes
  constexpr uint32_t ID64 = idesc_bf16(TROWS, NH), ID16 = idesc_bf16(TROWS, POUT);
  const uint64_t dX = mdesc(S.X, PIN), dH = mdesc(S.H, NH);
  const uint64_t dW1 = mdesc(S.W1, PIN), dW2 = mdesc(S.W2, NH), dW3 = mdesc(S.W3, NH), dW4 = mdesc(S.W4, NH);
  uint32_t phase = 0;
  bool ok = true;
  // one layer: MMAs over K (16 per instruction: 256 bytes = 16 descriptor
  // units further along K), commit, wait
  auto layer = [&](uint64_t da, uint64_t db, int ksteps, uint32_t dcol, uint32_t id) -> bool {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && !hold) {
      tc_fence_after();
      for (int kk = 0; kk < ksteps; ++kk)
        tc_mma(tmem + dcol, da + (uint64_t)(16 * kk), db + (uint64_t)(16 * kk), id, kk > 0 ? 1u : 0u);
      tc_commit(&S.mbar);
    }
    const bool w = mbar_wait(&S.mbar, phase);
    phase ^= 1u;
    tc_fence_after();
    return __syncthreads_and(w) != 0;
  };
  for (long long row0 = (long long)blockIdx.x * TROWS; row0 < n; row0 += (long long)gridDim.x * TROWS) {
    {
      const long long g = row0 + tid;
      float v[PIN];
#pragma unroll
      for (int k = 0; k < PIN; ++k) v[k] = (g < n && k < NIN) ? X[g * NIN + k] : 0.0f;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        *reinterpret_cast<uint4*>(S.X + cofs(tid, 8 * h, PIN)) =
            make_uint4(pack_bf16(v[8 * h], v[8 * h + 1]), pack_bf16(v[8 * h + 2], v[8 * h + 3]),
                       pack_bf16(v[8 * h + 4], v[8 * h + 5]), pack_bf16(v[8 * h + 6], v[8 * h + 7]));
    }
    if (!(ok = layer(dX, dW1, PIN / 16, 0, ID64))) break;
    tc_hidden(S, tl, S.b1);
    if (!(ok = layer(dH, dW2, NH / 16, 0, ID64))) break;
    tc_hidden(S, tl, S.b2);
    if (!(ok = layer(dH, dW3, NH / 16, 0, ID64))) break;
    tc_hidden(S, tl, S.b3);
    if (!(ok = layer(dH, dW4, NH / 16, NH, ID16))) break;
    uint32_t r[16];
    tmem_ld16(tl + (uint32_t)NH, r);
    tmem_wait_ld();
    const long long g = row0 + tid;
    if (g < n) {
#pragma unroll
      for (int j = 0; j < NOUT; ++j) Y[g * NOUT + j] = __uint_as_float(r[j]) + S.b4[j];
    }
  }
  if (!ok) {
    // a wait gave up: one more bounded wait for the MMAs still in flight
    (void)mbar_wait(&S.mbar, phase ^ 1u);
    if (tid == 0) atomicOr(status, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// sum of squared errors of pred against T over n rows, pred = network(X) or,
// with identity, the inputs' own HoT X[:, 5:13]; added to *acc
__global__ void __launch_bounds__(MT) k_mlp_loss(const float* __restrict__ p, const float* __restrict__ X,
                                                 const float* __restrict__ T, long long n, int identity,
                                                 double* __restrict__ acc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  __shared__ double s_acc;
  if (!identity) load_params(S, p);
  if (threadIdx.x == 0) s_acc = 0.0;
  __syncthreads();
  double local = 0.0;
  for (long long row0 = (long long)blockIdx.x * ROWS; row0 < n; row0 += (long long)gridDim.x * ROWS) {
    if (!identity) forward(S, X, row0, n);
    for (int i = threadIdx.x; i < ROWS * NOUT; i += MT) {
      const int r = i / NOUT, j = i % NOUT;
      const long long g = row0 + r;
      if (g < n) {
        const float y = identity ? X[g * NIN + 5 + j] : S.Y[r * POUT + j];
        const double e = (double)y - (double)T[g * NOUT + j];
        local += e * e;
      }
    }
    __syncthreads();
  }
  atomicAdd(&s_acc, local);
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(acc, s_acc);
}

// accumulate out[M x N] (FP32, rows < mrows, cols < ncols) into the gradient
// block at g (layout [m][ld])
__device__ void add_grad(const float* F, int N, int mrows, int ncols, float* g, int ld) {
  for (int i = threadIdx.x; i < mrows * N; i += MT) {
    const int j = i / N, k = i % N;
    if (k < ncols) atomicAdd(g + j * ld + k, F[i]);
  }
}

// forward + backward of mini-batch rows [b0, b0 + nb) of the row order perm
// (NULL: identity) over n_total rows; gradient of the batch loss
// 1/(8 nb) sum (y - t)^2 added to grad, sum of squared errors added to *loss.
// A perm entry outside [0, n_total) skips its row and sets *status.
__global__ void __launch_bounds__(MT) k_mlp_train(const float* __restrict__ p, const float* __restrict__ X,
                                                  const float* __restrict__ T, const int* __restrict__ perm,
                                                  long long n_total, long long b0, long long nb,
                                                  float* __restrict__ grad, double* __restrict__ loss,
                                                  int* __restrict__ status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  __shared__ float s_loss;
  __shared__ long long s_rows[ROWS];
  load_params(S, p);
  if (threadIdx.x == 0) s_loss = 0.0f;
  __syncthreads();
  const float scale = 2.0f / (float)(NOUT * nb);
  for (long long r0 = (long long)blockIdx.x * ROWS; r0 < nb; r0 += (long long)gridDim.x * ROWS) {
    // the rows of this tile (through the epoch's row order)
    for (int r = threadIdx.x; r < ROWS; r += MT) {
      long long g = -1;
      if (r0 + r < nb) {
        g = perm ? (long long)perm[b0 + r0 + r] : b0 + r0 + r;
        if (g < 0 || g >= n_total) {
          atomicOr(status, 1);
          g = -1;
        }
      }
      s_rows[r] = g;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * PIN; i += MT) {
      const int r = i / PIN, k = i % PIN;
      const long long g = s_rows[r];
      S.X[i] = __float2bfloat16_rn(g >= 0 && k < NIN ? X[g * NIN + k] : 0.0f);
    }
    __syncthreads();
    // forward (same as inference, inputs already staged)
    gemm_AWt<PIN, NH>(S.X, S.W1, S.F);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
      const float z = S.F[i] + S.b1[i % NH];
      S.A1[i] = __float2bfloat16_rn(gelu(z));
      S.G1[i] = gelu_d(z);
    }
    __syncthreads();
    gemm_AWt<NH, NH>(S.A1, S.W2, S.F);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
      const float z = S.F[i] + S.b2[i % NH];
      S.A2[i] = __float2bfloat16_rn(gelu(z));
      S.G2[i] = gelu_d(z);
    }
    __syncthreads();
    gemm_AWt<NH, NH>(S.A2, S.W3, S.F);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
      const float z = S.F[i] + S.b3[i % NH];
      S.A3[i] = __float2bfloat16_rn(gelu(z));
      S.G3[i] = gelu_d(z);
    }
    __syncthreads();
    gemm_AWt<NH, POUT>(S.A3, S.W4, S.Y);
    __syncthreads();
    // output delta (rows beyond the batch and padded outputs contribute 0)
    float lsum = 0.0f;
    for (int i = threadIdx.x; i < ROWS * POUT; i += MT) {
      const int r = i / POUT, j = i % POUT;
      const long long g = s_rows[r];
      float d = 0.0f;
      if (g >= 0 && j < NOUT) {
        const float e = S.Y[i] + S.b4[j] - T[g * NOUT + j];
        lsum += e * e;
        d = scale * e;
      }
      S.Y[i] = d;
      S.D4[i] = __float2bfloat16_rn(d);
    }
    atomicAdd(&s_loss, lsum);
    __syncthreads();
    // layer 4: dW4 = d4^T A3, db4, d3 = (d4 W4) . gelu'(z3)
    gemm_DtA<POUT, NH>(S.D4, S.A3, S.F);
    __syncthreads();
    add_grad(S.F, NH, NOUT, NH, grad + OFF_W4, NH);
    for (int j = threadIdx.x; j < NOUT; j += MT) {
      float s = 0.0f;
      for (int r = 0; r < ROWS; ++r) s += S.Y[r * POUT + j];
      atomicAdd(grad + OFF_B4 + j, s);
    }
    __syncthreads();
    gemm_DW<POUT, NH>(S.D4, S.W4, S.F);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
      const float d = S.F[i] * S.G3[i];
      S.F[i] = d;
      S.D[i] = __float2bfloat16_rn(d);
    }
    __syncthreads();
    // bias gradient of layer 3 (column sums of the FP32 delta)
    for (int j = threadIdx.x; j < NH; j += MT) {
      float s = 0.0f;
      for (int r = 0; r < ROWS; ++r) s += S.F[r * NH + j];
      atomicAdd(grad + OFF_B3 + j, s);
    }
    __syncthreads();
    gemm_DtA<NH, NH>(S.D, S.A2, S.F);
    __syncthreads();
    add_grad(S.F, NH, NH, NH, grad + OFF_W3, NH);
    __syncthreads();
    gemm_DW<NH, NH>(S.D, S.W3, S.F);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
      const float d = S.F[i] * S.G2[i];
      S.F[i] = d;
      S.D[i] = __float2bfloat16_rn(d);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NH; j += MT) {
      float s = 0.0f;
      for (int r = 0; r < ROWS; ++r) s += S.F[r * NH + j];
      atomicAdd(grad + OFF_B2 + j, s);
    }
    __syncthreads();
    gemm_DtA<NH, NH>(S.D, S.A1, S.F);
    __syncthreads();
    add_grad(S.F, NH, NH, NH, grad + OFF_W2, NH);
    __syncthreads();
    gemm_DW<NH, NH>(S.D, S.W2, S.F);
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * NH; i += MT) {
      const float d = S.F[i] * S.G1[i];
      S.F[i] = d;
      S.D[i] = __float2bfloat16_rn(d);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NH; j += MT) {
      float s = 0.0f;
      for (int r = 0; r < ROWS; ++r) s += S.F[r * NH + j];
      atomicAdd(grad + OFF_B1 + j, s);
    }
    __syncthreads();
    gemm_DtA<NH, PIN>(S.D, S.X, S.F);
    __syncthreads();
    add_grad(S.F, PIN, NH, NIN, grad + OFF_W1, NIN);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, (double)s_loss);
}

// Adam (Kingma and Ba 2015) on the FP32 master parameters; clears the gradient
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  g[i] = 0.0f;
}
}  // namespace

void launch_mlp_forward(const float* params, const float* X, long long n, float* Y, int* status, cudaStream_t s,
                        int hold) {
  if (n <= 0) return;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  long long nb = (n + TROWS - 1) / TROWS;
  if (nb > 4LL * sms) nb = 4LL * sms;
  k_mlp_forward_tc<<<(int)nb, TCT, TC_SMEM, s>>>(params, X, n, Y, status, hold);
  ++g_launches;
}

void launch_mlp_train_step(const float* params, const float* X, const float* T, const int* perm, long long n_total,
                           long long b0, long long nb, float* grad, double* loss, int* status, cudaStream_t s) {
  if (nb <= 0) return;
  const size_t sm = sizeof(Smem);
  cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  long long blocks = (nb + ROWS - 1) / ROWS;
  if (blocks > 304) blocks = 304;
  k_mlp_train<<<(int)blocks, MT, sm, s>>>(params, X, T, perm, n_total, b0, nb, grad, loss, status);
  ++g_launches;
}

void launch_mlp_loss(const float* params, const float* X, const float* T, long long n, int identity, double* acc,
                     cudaStream_t s) {
  if (n <= 0) return;
  const size_t sm = identity ? 0 : sizeof(Smem);
  cudaFuncSetAttribute(k_mlp_loss, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  long long blocks = (n + ROWS - 1) / ROWS;
  if (blocks > 608) blocks = 608;
  k_mlp_loss<<<(int)blocks, MT, sm, s>>>(params, X, T, n, identity, acc);
  ++g_launches;
}

void launch_adam(float* p, float* m, float* v, float* g, long long t, float lr, float b1, float b2, float eps,
                 cudaStream_t s) {
  const float c1 = (float)(1.0 - std::pow((double)b1, (double)t));
  const float c2 = (float)(1.0 - std::pow((double)b2, (double)t));
  k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(p, m, v, g, lr, b1, b2, eps, c1, c2);
  ++g_launches;
}

}  // namespace dig
