// dmr_noalloc.cu -- electron total of a density map without any device
// allocation by the library or the caller.
//
// Some callers cannot allocate device memory at all: a host application that
// hands every byte of the GPU to its own memory pool and forbids plug-ins to
// call cudaMalloc, code that runs inside a region where allocation is not
// permitted or would stall the device (cudaMalloc synchronises), or a caller
// that has no workspace to give.  For them this file keeps the reduction's
// scratch (one FP64 partial sum per thread block) in a fixed array that lives
// in the library's own device image.  The caller passes only the input map
// and the one-double output.
//
// The array is `g_partials` below: NOALLOC_MAX_BLOCKS doubles (128 KiB).  Every
// GPU that loads this library holds that much memory until the process exits.
// Each block reduces NOALLOC_NODES_PER_BLOCK nodes, so one call handles at most
// NOALLOC_MAX_BLOCKS * NOALLOC_NODES_PER_BLOCK nodes; larger maps are rejected.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "dmr.h"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_NODES_PER_THREAD = 16;
constexpr long long NOALLOC_NODES_PER_BLOCK = (long long)NOALLOC_THREADS * NOALLOC_NODES_PER_THREAD;
constexpr int NOALLOC_MAX_BLOCKS = 16384;

// Scratch of the reduction: one partial per block, rewritten by every call.
static __device__ __align__(256) double g_partials[NOALLOC_MAX_BLOCKS];

// Device address of g_partials per CUDA context, looked up once per context:
// the array's address belongs to the context that loaded the module, so a
// device reset (a new primary context) or a caller-made context needs a
// lookup of its own.  Contexts are told apart by the driver's unique context
// ID (a handle value can be reused after a context is destroyed).
constexpr int MAX_CONTEXTS = 64;
std::mutex g_mu;
struct Slot { unsigned long long ctx; double* ptr; };
Slot g_slots[MAX_CONTEXTS] = {};
int g_nslots = 0;

thread_local char g_msg[256] = "";

// Composite trapezoid weight of node (i, j) of an nx x ny cell mesh.
__device__ __forceinline__ double trap(int i, int j, int nx, int ny) {
  const double wx = (i == 0 || i == nx) ? 0.5 : 1.0;
  const double wy = (j == 0 || j == ny) ? 0.5 : 1.0;
  return wx * wy;
}

template <class T>
__global__ void k_total_partials(const T* __restrict__ n, int nx, int ny, long long nodes,
                                 double* partials) {
  __shared__ double sh[NOALLOC_THREADS / 32];
  const long long base = (long long)blockIdx.x * NOALLOC_NODES_PER_BLOCK;
  double acc = 0.0;
  for (int q = 0; q < NOALLOC_NODES_PER_THREAD; ++q) {
    const long long id = base + (long long)q * NOALLOC_THREADS + threadIdx.x;
    if (id < nodes) {
      const int j = (int)(id / (nx + 1)), i = (int)(id - (long long)j * (nx + 1));
      acc += trap(i, j, nx, ny) * (double)n[id];
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < NOALLOC_THREADS / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
}

__global__ void k_total_final(const double* partials, int nblk, double dx2, double* out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) acc += partials[q];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = dx2 * v;
  }
}

int fail(int code, const char* msg) {
  snprintf(g_msg, sizeof g_msg, "%s", msg);
  return code;
}

// The driver's cuCtxGetCurrent and cuCtxGetId, reached through the runtime
// (no link-time dependency on libcuda).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

void* driver_fn(const char* name) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return f;
}

// ID of the calling thread's current context; 0 when none is current.
int current_context(unsigned long long* out) {
  static CtxGetCurrentFn get = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get || !get_id) {
    get = reinterpret_cast<CtxGetCurrentFn>(driver_fn("cuCtxGetCurrent"));
    get_id = reinterpret_cast<CtxGetIdFn>(driver_fn("cuCtxGetId"));
    if (!get || !get_id) return fail(DMR_ECUDA, "cuCtxGetCurrent / cuCtxGetId are not available");
  }
  CUcontext c = nullptr;
  if (get(&c) != CUDA_SUCCESS) return fail(DMR_ECUDA, "cuCtxGetCurrent failed");
  *out = 0;
  if (c && get_id(c, out) != CUDA_SUCCESS) return fail(DMR_ECUDA, "cuCtxGetId failed");
  return DMR_OK;
}

// Device address of the scratch array in the current context.  The set-up
// (cudaGetSymbolAddress, with the caller's device current) runs on the first
// call made in each context; later calls in that context reuse the address.
int scratch_for_current_context(double** out) {
  std::lock_guard<std::mutex> lock(g_mu);   // also guards the driver entry points
  unsigned long long ctx = 0;
  if (int s = current_context(&ctx)) return s;
  if (ctx)
    for (int q = 0; q < g_nslots; ++q)
      if (g_slots[q].ctx == ctx) { *out = g_slots[q].ptr; return DMR_OK; }
  // the lookup also makes the runtime bind its context to this thread when
  // none was current yet
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
  if (e != cudaSuccess) return fail(DMR_ECUDA, cudaGetErrorString(e));
  if (!ctx)
    if (int s = current_context(&ctx)) return s;
  // a full table recycles its first entry (a context that ended long ago)
  const int q = g_nslots < MAX_CONTEXTS ? g_nslots++ : 0;
  g_slots[q] = Slot{ctx, static_cast<double*>(p)};
  *out = g_slots[q].ptr;
  return DMR_OK;
}

}  // namespace

extern "C" {

int dmr_electron_total_noalloc(const void* n_dev, int32_t nx, int32_t ny, int32_t precision,
                               double dx, void* cuda_stream, double* total_dev) {
  if (!n_dev || !total_dev) return fail(DMR_EINVAL, "null input or output pointer");
  if (nx < 1 || ny < 1 || !(dx > 0.0)) return fail(DMR_EINVAL, "nx, ny must be >= 1 and dx > 0");
  if (precision != 0 && precision != 1) return fail(DMR_EINVAL, "precision must be 0 or 1");
  // widened before the + 1, so nx or ny = INT32_MAX cannot overflow
  const long long nodes = ((long long)nx + 1) * ((long long)ny + 1);
  const long long max_nodes = (long long)NOALLOC_MAX_BLOCKS * NOALLOC_NODES_PER_BLOCK;
  if (nodes > max_nodes)
    return fail(DMR_ECAPACITY,
                "map larger than the fixed scratch allows (at most 67108864 nodes)");
  double* partials = nullptr;
  if (int s = scratch_for_current_context(&partials)) return s;
  const int nblk = (int)((nodes + NOALLOC_NODES_PER_BLOCK - 1) / NOALLOC_NODES_PER_BLOCK);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (precision == 1)
    k_total_partials<float><<<nblk, NOALLOC_THREADS, 0, st>>>((const float*)n_dev, nx, ny, nodes,
                                                              partials);
  else
    k_total_partials<double><<<nblk, NOALLOC_THREADS, 0, st>>>((const double*)n_dev, nx, ny,
                                                               nodes, partials);
  k_total_final<<<1, 1024, 0, st>>>(partials, nblk, dx * dx, total_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DMR_ECUDA, cudaGetErrorString(e));
  return DMR_OK;
}

const char* dmr_noalloc_last_error(void) { return g_msg; }

}  // extern "C"
