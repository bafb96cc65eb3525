// dig_sort.cu -- standalone stable counting sort of particles by cell (the
// paper's per-cell particle buckets, Sec. 4 / Listing 2, as a public op):
// cell[n] -> cell_start[n_cells+1] and order[] = indices of the kept elements
// sorted by cell, ties broken by index.  Entries outside [0, n_cells) are
// dropped (the removed-particle marker is -1).
//
//   count    histogram of cell ids (warp-aggregated atomics)
//   scan     cell_start = exclusive scan of the counts (two kernels)
//   place    order_tmp[cell_start[c] + atomic cursor] = i   (unordered in a cell)
//   fix      each cell's segment ranked by index: order[...] sorted
// Scratch (device, caller-provided): counts, cursors, scan partials, order_tmp.
#include "dig_internal.h"

namespace dig {

namespace {
constexpr int ST = 1024, SI = 4, SCH = ST * SI;

__host__ __device__ inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct SortScratch {
  int* counts;
  int* cursor;
  int* part;
  int* tmp;
};

__host__ __device__ inline SortScratch carve(char* base, long long n, int n_cells) {
  SortScratch s;
  size_t off = 0;
  s.counts = (int*)(base + off);
  off += al256(sizeof(int) * (size_t)n_cells);
  s.cursor = (int*)(base + off);
  off += al256(sizeof(int) * (size_t)n_cells);
  s.part = (int*)(base + off);
  off += al256(sizeof(int) * (size_t)((n_cells + SCH - 1) / SCH + 1));
  s.tmp = (int*)(base + off);
  return s;
}

__global__ void k_sort_zero(SortScratch S, int n_cells) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
    S.counts[c] = 0;
    S.cursor[c] = 0;
  }
}

__global__ void k_sort_count(const int* __restrict__ cell, long long n, int n_cells, SortScratch S) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = cell[i];
    if (c >= 0 && c < n_cells) atomicAdd(S.counts + c, 1);
  }
}

__global__ void __launch_bounds__(ST) k_sort_reduce(SortScratch S, int n_cells) {
  const int base = blockIdx.x * SCH;
  int t = 0;
  for (int i = threadIdx.x; i < SCH; i += ST)
    if (base + i < n_cells) t += S.counts[base + i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __shared__ int sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    t = sh[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) S.part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(ST) k_sort_scan(SortScratch S, int n_cells, int* __restrict__ cell_start) {
  __shared__ int sh[32];
  __shared__ int s_off;
  int p = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += ST) p += S.part[b];
  for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int w = 0; w < ST / 32; ++w) a += sh[w];
    s_off = a;
  }
  __syncthreads();
  const int c0 = blockIdx.x * SCH + threadIdx.x * SI;
  int v[SI], loc = 0;
#pragma unroll
  for (int i = 0; i < SI; ++i) {
    v[i] = c0 + i < n_cells ? S.counts[c0 + i] : 0;
    loc += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = loc;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = sh[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int e = s_off + inc - loc + (warp > 0 ? sh[warp - 1] : 0);
#pragma unroll
  for (int i = 0; i < SI; ++i) {
    const int c = c0 + i;
    if (c < n_cells) cell_start[c] = e;
    e += v[i];
    if (c == n_cells - 1) cell_start[n_cells] = e;
  }
}

__global__ void k_sort_place(const int* __restrict__ cell, long long n, int n_cells, const int* __restrict__ cs,
                             SortScratch S) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = cell[i];
    if (c >= 0 && c < n_cells) S.tmp[cs[c] + atomicAdd(S.cursor + c, 1)] = (int)i;
  }
}

// one warp per cell: rank each element of the segment by its index
__global__ void k_sort_fix(int n_cells, const int* __restrict__ cs, SortScratch S, int* __restrict__ order) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < n_cells; c += nw) {
    const int a = cs[c], len = cs[c + 1] - a;
    if (len <= 32) {
      const int key = lane < len ? S.tmp[a + lane] : 0x7fffffff;
      int r = 0;
      for (int q = 0; q < len; ++q) r += (__shfl_sync(0xffffffffu, key, q) < key) ? 1 : 0;
      if (lane < len) order[a + r] = key;
    } else {
      for (int k = lane; k < len; k += 32) {
        const int key = S.tmp[a + k];
        int r = 0;
        for (int q = 0; q < len; ++q) r += (S.tmp[a + q] < key) ? 1 : 0;
        order[a + r] = key;
      }
    }
  }
}
}  // namespace

size_t sort_scratch_bytes(long long n, int n_cells) {
  return al256(sizeof(int) * (size_t)n_cells) * 2 + al256(sizeof(int) * (size_t)((n_cells + SCH - 1) / SCH + 1)) +
         al256(sizeof(int) * (size_t)(n > 0 ? n : 1));
}

void launch_sort_by_cell(const int* cell, long long n, int n_cells, int* cell_start, int* order, char* scratch,
                         cudaStream_t s) {
  const SortScratch S = carve(scratch, n, n_cells);
  const int nb = (n_cells + SCH - 1) / SCH;
  const int gridc = (int)((n_cells + 255) / 256 < 4096 ? (n_cells + 255) / 256 : 4096);
  const int gridn = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  k_sort_zero<<<gridc > 0 ? gridc : 1, 256, 0, s>>>(S, n_cells);
  if (n > 0) k_sort_count<<<gridn, 256, 0, s>>>(cell, n, n_cells, S);
  k_sort_reduce<<<nb, ST, 0, s>>>(S, n_cells);
  k_sort_scan<<<nb, ST, 0, s>>>(S, n_cells, cell_start);
  if (n > 0) {
    k_sort_place<<<gridn, 256, 0, s>>>(cell, n, n_cells, cell_start, S);
    const int gw = (n_cells + 7) / 8 < 8192 ? (n_cells + 7) / 8 : 8192;
    k_sort_fix<<<gw, 256, 0, s>>>(n_cells, cell_start, S, order);
  }
  g_launches += n > 0 ? 6 : 4;
}

}  // namespace dig
