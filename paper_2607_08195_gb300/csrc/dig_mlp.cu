// dig_mlp.cu -- learned per-cell closure: MLP 13 -> 64 -> 64 -> 64 -> 8 with
// GELU, BF16 weights and activations, FP32 accumulation, on the
// fifth-generation tensor cores (tcgen05.mma with FP32 accumulators in
// tensor memory, 128 rows per tile).  Inference (S12: the coupling's closure,
// closure_forward and the loss): k_mlp_forward_tc.  Training (S13): forward
// and backward with the weight gradients dW = delta^T A accumulated in
// tensor memory (k_mlp_train_tc); Adam on the FP32 master parameters.
//
// Parameter layout (FP32 master, [out][in] per layer): W1[64][13] b1[64]
// W2[64][64] b2[64] W3[64][64] b3[64] W4[8][64] b4[8].  In shared memory the
// weights are BF16 [out][in] with the input dimension of layer 1 padded to 16
// and the outputs of layer 4 padded to 16 (zeros).
#include "dig_internal.h"

#include <cuda_bf16.h>

namespace dig {

namespace {
constexpr int NIN = 13, NH = 64, NOUT = 8, PIN = 16, POUT = 16;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH, OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + NOUT * NH,
              NPARAM = OFF_B4 + NOUT;
static_assert(NPARAM == 9736, "parameter count");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678f)) + z * expf(-0.5f * z * z) * 0.39894228f;
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

// With T non-null the squared errors of the outputs against T[n][8] are
// summed (FP64) into *acc instead of (or besides) writing Y.
__global__ void __launch_bounds__(TCT) k_mlp_forward_tc(const float* __restrict__ p, const float* __restrict__ X,
                                                       long long n, float* __restrict__ Y,
                                                       const float* __restrict__ T, double* __restrict__ acc,
                                                       int* __restrict__ status, int hold) {
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
  double lsq = 0.0;
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
      for (int j = 0; j < NOUT; ++j) {
        const float y = __uint_as_float(r[j]) + S.b4[j];
        if (Y) Y[g * NOUT + j] = y;
        if (T) {
          const double e = (double)y - (double)T[g * NOUT + j];
          lsq += e * e;
        }
      }
    }
  }
  if (T) {
    for (int o = 16; o > 0; o >>= 1) lsq += __shfl_xor_sync(0xffffffffu, lsq, o);
    if ((tid & 31) == 0) atomicAdd(acc, lsq);
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

// ---------------------------------------------------------------------------
// Training step on tcgen05 (forward and backward of tiles of 128 rows: BF16
// operands, FP32 accumulators, FP32 deltas for the bias gradients).  Every GEMM has
// M = 128: the forward and the delta propagation run over the tile's rows; a
// weight gradient dW = delta^T A contracts over the rows, so its operands are
// the transposed delta (out x rows, padded to 128 output rows whose results
// are ignored) and the transposed activations (in x rows), both written
// K-major by the epilogues.  The weight gradients accumulate in TMEM over the
// CTA's tiles and are added to the global gradient once.  The
// pre-activations needed for GELU' are recomputed by the same MMAs as in the
// forward (identical values) instead of being kept.  Eight warps: warp w
// reads TMEM lanes 32 (w mod 4) .. +31 (the rows) and the column half w / 4,
// so each thread's epilogue covers 32 of a row's 64 values.
// TMEM columns: [0,64) and [64,128) scratch, [128,144) the output layer,
// [144,160) dW1, [160,224) dW2, [224,288) dW3, [288,352) dW4.
// ---------------------------------------------------------------------------
constexpr uint32_t TR_COLS = 512;
constexpr int RT = 128;   // rows of the transposed operands (the contraction dimension)
constexpr int TRT = 256;  // threads of the training CTA
constexpr int HC = NH / 2;

struct TrSmem {
  alignas(128) __nv_bfloat16 W1[NH * PIN];
  alignas(128) __nv_bfloat16 W2[NH * NH];
  alignas(128) __nv_bfloat16 W3[NH * NH];
  alignas(128) __nv_bfloat16 W4[POUT * NH];
  alignas(128) __nv_bfloat16 W2T[NH * NH];    // [in][out] of layer 2 (B of the delta propagation)
  alignas(128) __nv_bfloat16 W3T[NH * NH];
  alignas(128) __nv_bfloat16 W4T[NH * POUT];  // [in 64][out 16]
  alignas(128) __nv_bfloat16 X[TROWS * PIN];
  alignas(128) __nv_bfloat16 A1[TROWS * NH];
  alignas(128) __nv_bfloat16 A2[TROWS * NH];
  alignas(128) __nv_bfloat16 A3[TROWS * NH];
  alignas(128) __nv_bfloat16 XT[PIN * RT];    // [16][128]
  alignas(128) __nv_bfloat16 A1T[NH * RT];    // [64][128]
  alignas(128) __nv_bfloat16 A2T[NH * RT];
  alignas(128) __nv_bfloat16 A3T[NH * RT];
  alignas(128) __nv_bfloat16 D[TROWS * NH];   // delta of the current layer, [128 rows][64]
  alignas(128) __nv_bfloat16 D4[TROWS * POUT];
  alignas(128) __nv_bfloat16 DT[RT * RT];     // [out, padded to 128][128 rows]
  float b1[NH], b2[NH], b3[NH], b4[POUT];
  float tgt[TROWS * NOUT];                    // targets of the tile's rows
  long long rows[TROWS];
  float red[TRT / 32];
  alignas(8) unsigned long long mbar;
  uint32_t tmem;
};
constexpr size_t TR_SMEM = sizeof(TrSmem);
static_assert(sizeof(TrSmem) <= 227 * 1024, "tcgen05 training shared memory");

// 32 FP32 accumulator columns of the thread's row at tl + col
__device__ __forceinline__ void tmem_row32(uint32_t tl, uint32_t col, float (&v)[HC]) {
#pragma unroll
  for (int c = 0; c < HC; c += 16) {
    uint32_t r[16];
    tmem_ld16(tl + col + (uint32_t)c, r);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[c + i] = __uint_as_float(r[i]);
  }
}

// columns [c0, c0 + 32) of row `row` of an operand with K = 64 (K-major), BF16
__device__ __forceinline__ void put_row32(__nv_bfloat16* buf, int row, int c0, const float (&a)[HC]) {
#pragma unroll
  for (int h = 0; h < HC / 8; ++h)
    *reinterpret_cast<uint4*>(buf + cofs(row, c0 + 8 * h, NH)) =
        make_uint4(pack_bf16(a[8 * h], a[8 * h + 1]), pack_bf16(a[8 * h + 2], a[8 * h + 3]),
                   pack_bf16(a[8 * h + 4], a[8 * h + 5]), pack_bf16(a[8 * h + 6], a[8 * h + 7]));
}

// entries [c0, c0 + M) of column `row` of a transposed operand [m][128 rows]
template <int M>
__device__ __forceinline__ void put_col(__nv_bfloat16* buf, int row, int c0, const float* a) {
#pragma unroll
  for (int j = 0; j < M; ++j) buf[cofs(c0 + j, row, RT)] = __float2bfloat16_rn(a[j]);
}

// sum over the warp's 32 rows of each of the thread's values, added to g[j]
template <int M>
__device__ __forceinline__ void bias_grad(const float* d, float* g, int lane) {
#pragma unroll
  for (int j = 0; j < M; ++j) {
    float t = d[j];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) atomicAdd(g + j, t);
  }
}

__global__ void __launch_bounds__(TRT) k_mlp_train_tc(const float* __restrict__ p, const float* __restrict__ X,
                                                     const float* __restrict__ T, const int* __restrict__ perm,
                                                     long long n_total, long long b0, long long nb,
                                                     float* __restrict__ grad, double* __restrict__ loss,
                                                     int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TrSmem& S = *reinterpret_cast<TrSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = 32 * (warp & 3) + lane, half = warp >> 2, c0 = HC * half;
  // weights (forward and transposed) and biases
  for (int i = tid; i < NH * PIN; i += TRT) {
    const int j = i / PIN, k = i % PIN;
    S.W1[cofs(j, k, PIN)] = __float2bfloat16_rn(k < NIN ? p[OFF_W1 + j * NIN + k] : 0.0f);
  }
  for (int i = tid; i < NH * NH; i += TRT) {
    const int j = i / NH, k = i % NH;
    const __nv_bfloat16 w2 = __float2bfloat16_rn(p[OFF_W2 + i]), w3 = __float2bfloat16_rn(p[OFF_W3 + i]);
    S.W2[cofs(j, k, NH)] = w2;
    S.W3[cofs(j, k, NH)] = w3;
    S.W2T[cofs(k, j, NH)] = w2;
    S.W3T[cofs(k, j, NH)] = w3;
  }
  for (int i = tid; i < POUT * NH; i += TRT) {
    const int j = i / NH, k = i % NH;
    const __nv_bfloat16 w4 = __float2bfloat16_rn(j < NOUT ? p[OFF_W4 + i] : 0.0f);
    S.W4[cofs(j, k, NH)] = w4;
    S.W4T[cofs(k, j, POUT)] = w4;
  }
  for (int i = tid; i < NH; i += TRT) {
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
                 "r"(TR_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t tl = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's 32 lanes (rows)
  constexpr uint32_t ID64 = idesc_bf16(TROWS, NH), ID16 = idesc_bf16(TROWS, POUT);
  constexpr uint32_t C_S1 = 0, C_S2 = 64, C_Y = 128, C_W1 = 144, C_W2 = 160, C_W3 = 224, C_W4 = 288;
  const uint64_t dX = mdesc(S.X, PIN), dA1 = mdesc(S.A1, NH), dA2 = mdesc(S.A2, NH), dA3 = mdesc(S.A3, NH);
  const uint64_t dW1 = mdesc(S.W1, PIN), dW2 = mdesc(S.W2, NH), dW3 = mdesc(S.W3, NH), dW4 = mdesc(S.W4, NH);
  const uint64_t dW2T = mdesc(S.W2T, NH), dW3T = mdesc(S.W3T, NH), dW4T = mdesc(S.W4T, POUT);
  const uint64_t dXT = mdesc(S.XT, RT), dA1T = mdesc(S.A1T, RT), dA2T = mdesc(S.A2T, RT), dA3T = mdesc(S.A3T, RT);
  const uint64_t dD = mdesc(S.D, NH), dD4 = mdesc(S.D4, POUT), dDT = mdesc(S.DT, RT);
  uint32_t phase = 0;
  bool ok = true;
  int tiles = 0;
  // MMAs issued by one thread: (a, b, k-steps, TMEM column, instruction
  // descriptor, accumulate into the column's previous contents)
  struct Op {
    uint64_t a, b;
    int ks;
    uint32_t col, id;
    bool acc;
  };
  auto issue = [&](const Op* ops, int nops) -> bool {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int o = 0; o < nops; ++o)
        for (int kk = 0; kk < ops[o].ks; ++kk)
          tc_mma(tmem + ops[o].col, ops[o].a + (uint64_t)(16 * kk), ops[o].b + (uint64_t)(16 * kk), ops[o].id,
                 (ops[o].acc || kk > 0) ? 1u : 0u);
      tc_commit(&S.mbar);
    }
    const bool w = mbar_wait(&S.mbar, phase);
    phase ^= 1u;
    tc_fence_after();
    return __syncthreads_and(w) != 0;
  };
  const float scale = 2.0f / (float)(NOUT * nb);
  float lsum = 0.0f;
  for (long long r0 = (long long)blockIdx.x * TROWS; r0 < nb && ok; r0 += (long long)gridDim.x * TROWS) {
    const bool acc = tiles > 0;
    // the tile's rows through the epoch's row order, inputs and targets
    if (half == 0) {
      long long g = -1;
      if (r0 + row < nb) {
        g = perm ? (long long)perm[b0 + r0 + row] : b0 + r0 + row;
        if (g < 0 || g >= n_total) {
          atomicOr(status, 1);
          g = -1;
        }
      }
      S.rows[row] = g;
      float v[PIN];
#pragma unroll
      for (int k = 0; k < PIN; ++k) v[k] = (g >= 0 && k < NIN) ? X[g * NIN + k] : 0.0f;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        *reinterpret_cast<uint4*>(S.X + cofs(row, 8 * h, PIN)) =
            make_uint4(pack_bf16(v[8 * h], v[8 * h + 1]), pack_bf16(v[8 * h + 2], v[8 * h + 3]),
                       pack_bf16(v[8 * h + 4], v[8 * h + 5]), pack_bf16(v[8 * h + 6], v[8 * h + 7]));
      put_col<PIN>(S.XT, row, 0, v);
#pragma unroll
      for (int j = 0; j < NOUT; ++j) S.tgt[row * NOUT + j] = g >= 0 ? T[g * NOUT + j] : 0.0f;
    }
    // forward
    float z[HC], a[HC];
    for (int l = 0; l < 3 && ok; ++l) {
      const uint64_t fin = l == 0 ? dX : l == 1 ? dA1 : dA2, fw = l == 0 ? dW1 : l == 1 ? dW2 : dW3;
      const float* bl = l == 0 ? S.b1 : l == 1 ? S.b2 : S.b3;
      __nv_bfloat16* Al = l == 0 ? S.A1 : l == 1 ? S.A2 : S.A3;
      __nv_bfloat16* ATl = l == 0 ? S.A1T : l == 1 ? S.A2T : S.A3T;
      const Op op = {fin, fw, l == 0 ? PIN / 16 : NH / 16, C_S1, ID64, false};
      if (!(ok = issue(&op, 1))) break;
      tmem_row32(tl, C_S1 + (uint32_t)c0, z);
#pragma unroll
      for (int j = 0; j < HC; ++j) a[j] = gelu(z[j] + bl[c0 + j]);
      put_row32(Al, row, c0, a);
      put_col<HC>(ATl, row, c0, a);
    }
    if (!ok) break;
    {
      const Op op = {dA3, dW4, NH / 16, C_Y, ID16, false};
      if (!(ok = issue(&op, 1))) break;
    }
    // output delta (FP32) and its BF16 copies; loss (the first column half)
    float d[HC];
    if (half == 0) {
      uint32_t r[16];
      tmem_ld16(tl + C_Y, r);
      tmem_wait_ld();
      const bool live = S.rows[row] >= 0;
#pragma unroll
      for (int j = 0; j < NOUT; ++j) {
        d[j] = 0.0f;
        if (live) {
          const float e = __uint_as_float(r[j]) + S.b4[j] - S.tgt[row * NOUT + j];
          lsum += e * e;
          d[j] = scale * e;
        }
      }
      *reinterpret_cast<uint4*>(S.D4 + cofs(row, 0, POUT)) =
          make_uint4(pack_bf16(d[0], d[1]), pack_bf16(d[2], d[3]), pack_bf16(d[4], d[5]), pack_bf16(d[6], d[7]));
      *reinterpret_cast<uint4*>(S.D4 + cofs(row, 8, POUT)) = make_uint4(0u, 0u, 0u, 0u);
      put_col<NOUT>(S.DT, row, 0, d);
      bias_grad<NOUT>(d, grad + OFF_B4, lane);
    }
    // backward: per layer l = 3, 2, 1 the weight gradient of layer l + 1, the
    // delta propagated through it and the recomputed pre-activation of layer l
    for (int s = 0; s < 3 && ok; ++s) {
      const uint64_t bW = s == 0 ? dA3T : s == 1 ? dA2T : dA1T;
      const uint32_t cW = s == 0 ? C_W4 : s == 1 ? C_W3 : C_W2;
      const uint64_t bT = s == 0 ? dW4T : s == 1 ? dW3T : dW2T;
      const uint64_t aP = s == 0 ? dD4 : dD;
      const uint64_t zi = s == 0 ? dA2 : s == 1 ? dA1 : dX, zw = s == 0 ? dW3 : s == 1 ? dW2 : dW1;
      const float* zb = s == 0 ? S.b3 : s == 1 ? S.b2 : S.b1;
      float* gb = grad + (s == 0 ? OFF_B3 : s == 1 ? OFF_B2 : OFF_B1);
      const Op ops[3] = {{dDT, bW, RT / 16, cW, ID64, acc},
                         {aP, bT, s == 0 ? POUT / 16 : NH / 16, C_S1, ID64, false},
                         {zi, zw, s == 2 ? PIN / 16 : NH / 16, C_S2, ID64, false}};
      if (!(ok = issue(ops, 3))) break;
      float pre[HC];
      tmem_row32(tl, C_S1 + (uint32_t)c0, pre);
      tmem_row32(tl, C_S2 + (uint32_t)c0, z);
#pragma unroll
      for (int j = 0; j < HC; ++j) d[j] = pre[j] * gelu_d(z[j] + zb[c0 + j]);
      if (s < 2) put_row32(S.D, row, c0, d);
      put_col<HC>(S.DT, row, c0, d);
      bias_grad<HC>(d, gb + c0, lane);
    }
    if (!ok) break;
    {
      const Op op = {dDT, dXT, RT / 16, C_W1, idesc_bf16(TROWS, PIN), acc};
      if (!(ok = issue(&op, 1))) break;
    }
    ++tiles;
  }
  // loss of the CTA's rows
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) S.red[warp] = lsum;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
    for (int w = 0; w < TRT / 32; ++w) t += S.red[w];
    atomicAdd(loss, (double)t);
  }
  // the weight gradients accumulated over the CTA's tiles: output row j in
  // TMEM lane j (warps 0, 1, 4, 5; layer 4's eight rows in warps 0 and 4),
  // each warp its column half
  if (ok && tiles > 0 && (warp & 3) < 2) {
    const int j = row;
    float v[HC];
    tmem_row32(tl, C_W2 + (uint32_t)c0, v);
    for (int k = 0; k < HC; ++k) atomicAdd(grad + OFF_W2 + j * NH + c0 + k, v[k]);
    tmem_row32(tl, C_W3 + (uint32_t)c0, v);
    for (int k = 0; k < HC; ++k) atomicAdd(grad + OFF_W3 + j * NH + c0 + k, v[k]);
    tmem_row32(tl, C_W4 + (uint32_t)c0, v);
    if (j < NOUT)
      for (int k = 0; k < HC; ++k) atomicAdd(grad + OFF_W4 + j * NH + c0 + k, v[k]);
    if (half == 0) {
      uint32_t r[16];
      tmem_ld16(tl + C_W1, r);
      tmem_wait_ld();
      for (int k = 0; k < NIN; ++k) atomicAdd(grad + OFF_W1 + j * NIN + k, __uint_as_float(r[k]));
    }
  }
  if (!ok) {
    (void)mbar_wait(&S.mbar, phase ^ 1u);
    if (tid == 0) atomicOr(status, 2);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TR_COLS) : "memory");
  }
}

// sum of squared errors of the inputs' own HoT X[:, 5:13] against T over n
// rows (the closure without the network), added to *acc
__global__ void k_mlp_loss_identity(const float* __restrict__ X, const float* __restrict__ T, long long n,
                                    double* __restrict__ acc) {
  double local = 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x)
    for (int j = 0; j < NOUT; ++j) {
      const double e = (double)X[g * NIN + 5 + j] - (double)T[g * NOUT + j];
      local += e * e;
    }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, local);
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
                        int hold, const float* T, double* acc) {
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
  k_mlp_forward_tc<<<(int)nb, TCT, TC_SMEM, s>>>(params, X, n, Y, T, acc, status, hold);
  ++g_launches;
}

void launch_mlp_train_step(const float* params, const float* X, const float* T, const int* perm, long long n_total,
                           long long b0, long long nb, float* grad, double* loss, int* status, cudaStream_t s) {
  if (nb <= 0) return;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
  }
  cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM);
  long long blocks = (nb + TROWS - 1) / TROWS;
  if (blocks > sms) blocks = sms;  // one CTA per SM: its tiles' weight gradients accumulate in its TMEM
  k_mlp_train_tc<<<(int)blocks, TRT, TR_SMEM, s>>>(params, X, T, perm, n_total, b0, nb, grad, loss, status);
  ++g_launches;
}

void launch_mlp_loss(const float* params, const float* X, const float* T, long long n, int identity, double* acc,
                     int* status, cudaStream_t s) {
  if (n <= 0) return;
  if (identity) {
    long long blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    k_mlp_loss_identity<<<(int)blocks, 256, 0, s>>>(X, T, n, acc);
    ++g_launches;
    return;
  }
  launch_mlp_forward(params, X, n, nullptr, status, s, 0, T, acc);
}

void launch_adam(float* p, float* m, float* v, float* g, long long t, float lr, float b1, float b2, float eps,
                 cudaStream_t s) {
  const float c1 = (float)(1.0 - std::pow((double)b1, (double)t));
  const float c2 = (float)(1.0 - std::pow((double)b2, (double)t));
  k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(p, m, v, g, lr, b1, b2, eps, c1, c2);
  ++g_launches;
}

}  // namespace dig
