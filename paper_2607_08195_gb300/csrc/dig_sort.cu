// dig_sort.cu -- standalone stable counting sort of particles by cell (the
// paper's per-cell particle buckets, Sec. 4 / Listing 2, as a public op):
// cell[n] -> cell_start[n_cells+1] and order[] = indices of the kept elements
// sorted by cell, ties broken by index.  Entries outside [0, n_cells) are
// dropped (the removed-particle marker is -1).
//
//   count    histogram of cell ids (warp-aggregated atomics)
//   scan     cell_start = exclusive scan of the counts (two kernels)
//   place    order_tmp[cell_start[c] + atomic cursor] = i   (unordered in a cell)
//   fix      each cell's segment ordered by index: warp ranking up to 32
//            elements, a block's stable radix sort beyond (linear time)
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

// one warp per cell: segments of up to 32 elements ranked by index within
// the warp; longer segments are left to k_sort_long
__global__ void k_sort_fix(int n_cells, const int* __restrict__ cs, SortScratch S, int* __restrict__ order) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < n_cells; c += nw) {
    const int a = cs[c], len = cs[c + 1] - a;
    if (len > 32) continue;
    const int key = lane < len ? S.tmp[a + lane] : 0x7fffffff;
    int r = 0;
    for (int q = 0; q < len; ++q) r += (__shfl_sync(0xffffffffu, key, q) < key) ? 1 : 0;
    if (lane < len) order[a + r] = key;
  }
}

// Segments longer than 32: one block per segment, a stable LSD radix sort of
// its keys (distinct indices) by 8-bit digits, as many passes as the largest
// key needs, ping-ponging between tmp and order over the segment's own range;
// each pass counts the digits, scans them, then places the keys tile by tile
// in index order (rank within a tile: lanes with the same digit in earlier
// warps, then earlier lanes of the same warp).  Work O(len) per pass.
constexpr int LT = 256, LW = LT / 32;

__global__ void __launch_bounds__(LT) k_sort_long(int n_cells, const int* __restrict__ cs, SortScratch S,
                                                 int* __restrict__ order) {
  __shared__ int hist[256], off[256], wcnt[LW][256];
  __shared__ int s_max;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int c = blockIdx.x; c < n_cells; c += gridDim.x) {
    const int a = cs[c], len = cs[c + 1] - a;
    if (len <= 32) continue;  // block-uniform
    // the largest key fixes the number of passes
    int mx = 0;
    for (int k = t; k < len; k += LT) mx = max(mx, S.tmp[a + k]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (t == 0) s_max = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_max, mx);
    __syncthreads();
    int bits = 0;
    while (bits < 31 && (s_max >> bits) != 0) bits += 8;
    const int passes = bits > 0 ? bits / 8 : 1;
    int* src = S.tmp + a;
    int* dst = order + a;
    for (int p = 0; p < passes; ++p) {
      const int sh = 8 * p;
      hist[t] = 0;
      __syncthreads();
      for (int k = t; k < len; k += LT) atomicAdd(&hist[(src[k] >> sh) & 255], 1);
      __syncthreads();
      if (warp == 0) {  // exclusive scan of the 256 counts, 8 per lane
        int v[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          v[i] = hist[8 * lane + i];
          sum += v[i];
        }
        int inc = sum;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        int e = inc - sum;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          off[8 * lane + i] = e;
          e += v[i];
        }
      }
      __syncthreads();
      for (int k0 = 0; k0 < len; k0 += LT) {
        const int k = k0 + t;
        const bool in = k < len;
        const int key = in ? src[k] : 0;
        const int d = in ? (key >> sh) & 255 : 256 + t;  // out-of-range lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int below = __popc(peers & ((1u << lane) - 1u));
        for (int i = t; i < LW * 256; i += LT) wcnt[i / 256][i % 256] = 0;
        __syncthreads();
        if (in && below == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (in) {
          int r = off[d] + below;
          for (int w = 0; w < warp; ++w) r += wcnt[w][d];
          dst[r] = key;
        }
        __syncthreads();
        // advance each digit's offset by its count in this tile
        int tot = 0;
        for (int w = 0; w < LW; ++w) tot += wcnt[w][t];
        off[t] += tot;
        __syncthreads();
      }
      int* x = src;
      src = dst;
      dst = x;
      __syncthreads();
    }
    if (src != order + a)  // an even number of passes left the result in tmp
      for (int k = t; k < len; k += LT) order[a + k] = src[k];
    __syncthreads();
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
    k_sort_long<<<n_cells < 1024 ? n_cells : 1024, LT, 0, s>>>(n_cells, cell_start, S, order);
  }
  g_launches += n > 0 ? 7 : 4;
}

}  // namespace dig
