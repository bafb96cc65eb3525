// dig_noalloc.cu -- an allocation-free variant of dig_sort_by_cell.
//
// Some callers cannot allocate device memory at all: code that runs inside a
// host framework which owns every device allocation (a custom allocator that
// hands out only the buffers it planned), a plug-in called from a real-time
// loop where cudaMalloc's implicit device synchronisation is not allowed, or a
// process that has reached a hard memory budget.  Such a caller can still
// provide its inputs and outputs, but not the working memory that
// dig_sort_by_cell asks for.  This variant takes its working memory from one
// fixed array compiled into the library instead.
//
// The working memory is a file-scope __device__ array of
// DIG_NOALLOC_SCRATCH_BYTES: every GPU that loads the library keeps it until
// the process exits.  It is shared by all calls, which therefore must not
// overlap on the GPU (two calls in flight at once, on different streams or
// from different threads, race on it).  The kernels clear the counters they
// need at the start of every call; everything else in the array is
// overwritten before it is read.
//
// The device address of the array is looked up with cudaGetSymbolAddress on
// every call, for the device current at the call (host code cannot use the
// array's name as a device address).  The lookup is a cheap host call once the
// module is loaded on that device, and it stays right if the context is
// destroyed and made again (cudaDeviceReset), which can move the array.  The
// first call on a device loads the module there: make it before capturing
// any stream on that device.
#include "../../include/dig.h"
#include "dig_internal.h"

namespace dig {

static __device__ __align__(256) unsigned char g_sort_scratch[DIG_NOALLOC_SCRATCH_BYTES];

namespace {
// failures are reported like the other context-free calls: dig_last_error(NULL)
int noalloc_fail(int code, const char* msg) {
  set_thread_error(msg);
  return code;
}

// device address of g_sort_scratch on the current device
int scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (e != cudaSuccess || !p) return noalloc_fail(DIG_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
  *out = p;
  return DIG_OK;
}
}  // namespace

}  // namespace dig

extern "C" int dig_sort_by_cell_noalloc(const int32_t* cell, int64_t n, int32_t n_cells, int32_t* cell_start,
                                        int32_t* order, void* stream) {
  using namespace dig;
  if (n < 0 || n_cells <= 0 || !cell_start || (n > 0 && (!cell || !order)))
    return noalloc_fail(DIG_ERR_ARG, "dig_sort_by_cell_noalloc: bad arguments");
  if (n > DIG_NOALLOC_MAX_N || n_cells > DIG_NOALLOC_MAX_CELLS)
    return noalloc_fail(DIG_ERR_CAPACITY,
                        "dig_sort_by_cell_noalloc: n or n_cells above the fixed scratch limits "
                        "(DIG_NOALLOC_MAX_N, DIG_NOALLOC_MAX_CELLS); use dig_sort_by_cell");
  if (sort_scratch_bytes(n, n_cells) > (size_t)DIG_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(DIG_ERR_CAPACITY, "dig_sort_by_cell_noalloc: scratch limit exceeded");
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  launch_sort_by_cell(cell, n, n_cells, cell_start, order, (char*)scratch, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(DIG_ERR_CUDA, cudaGetErrorString(e));
  return DIG_OK;
}
