// rvea_select_noalloc: environmental selection for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they want a selection: code running under a fixed, pre-planned device
// memory budget (an inference-server or plugin execution step, where the
// host framework owns every byte and forbids allocation while work is being
// enqueued), or code whose device memory is entirely reserved by another
// framework's caching allocator.  For them this file keeps the scratch that
// rvea_select would take from the caller in a file-scope device array of a
// fixed maximum size.  The array belongs to this file's GPU module: under
// CUDA's lazy module loading (the default) the module, and with it the
// array, is loaded on a device by the first call there (the address lookup
// below); with CUDA_MODULE_LOADING=EAGER it is loaded with the library's
// other modules when the process first uses the device.  Either way a later
// call maps nothing new, and no call asks an allocator for memory: the
// descriptor and the work-item table are written by a kernel straight from
// its parameters, with no host-side buffer.
//
// The same kernels as rvea_select run on that array, so results are the same
// bit for bit.  Every call shares the one array: two calls whose work
// overlaps on the GPU (different streams, no ordering between them) race and
// corrupt each other's results; calls on one stream, or otherwise ordered,
// are safe.  The array keeps the previous call's contents; every field a
// call reads is cleared by the call itself before use.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/rvea.h"
#include "rvea_device.cuh"

namespace rvea {
__global__ void k_select(const __grid_constant__ BatchDir dir);
__global__ void k_op_prep(const RunDesc *Rp);
__global__ void k_op_zstar(const RunDesc *Rp);
__global__ void k_op_finish(const RunDesc *Rp);
}  // namespace rvea

using namespace rvea;

namespace {

constexpr size_t kNoAllocBytes = size_t(4) << 20;   // 4 MiB per device
constexpr int kNoAllocMaxN = 65536;                  // solutions
constexpr int kNoAllocMaxR = 16384;                  // reference vectors
constexpr int kDevicesMax = 64;

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_select_scratch[kNoAllocBytes];

// Writes the run descriptor and the full-scan work items into the scratch,
// and the zero-padded float4 rows of V, from the kernel's parameters.
__global__ void k_noalloc_setup(const __grid_constant__ RunDesc D, RunDesc *out, SelItem *items,
                                int nblk, int nch, int chunk, const float *V, float *V32) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  if (tid == 0) *out = D;
  const int r = D.N, m = D.m, w = 4 * D.m4;
  for (int q = tid; q < nblk * nch; q += nth) {
    const int b = q / nch, c = q - b * nch;
    items[q] = SelItem{b, min(r, c * chunk), min(r, (c + 1) * chunk), nch};
  }
  for (int q = tid; q < r * w; q += nth) {
    const int j = q / w, k = q - j * w;
    V32[q] = k < m ? V[(size_t)j * m + k] : 0.0f;
  }
}

std::mutex g_mu;
void *g_scratch_addr[kDevicesMax] = {};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carve {
  size_t ctl, desc, best, amax, blk, items, v32, total;
};

Carve carve(int n, int r, int m, int n_items) {
  Carve c;
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = up256(o + b);
    return at;
  };
  const int nblk = (n + kSelBlock - 1) / kSelBlock;
  c.ctl = take(sizeof(Ctl));
  c.desc = take(sizeof(RunDesc));
  c.best = take((size_t)r * 8);
  c.amax = take((size_t)n * 8);
  c.blk = take((size_t)nblk * 4);
  c.items = take((size_t)n_items * sizeof(SelItem));
  c.v32 = take((size_t)r * ((m + 3) / 4) * 16);
  c.total = o;
  return c;
}

// Device address of the scratch on the current device, looked up once per
// device (with that device current).  The same one-time set-up lets the
// selection kernel use more than 48 KB of dynamic shared memory (needed for
// m > 8), as the other entry points do on their first call.
rvea_status scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevicesMax) return RVEA_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return RVEA_ERR_CUDA;
    }
    int optin = 0;
    cudaFuncAttributes fa;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, (const void *)k_select) != cudaSuccess ||
        cudaFuncSetAttribute((const void *)k_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
      cudaGetLastError();
      return RVEA_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
  return RVEA_OK;
}

}  // namespace

extern "C" {

rvea_status rvea_select_noalloc(int m, int n, const float *F, const uint8_t *valid, int r,
                                const float *V, const float *gamma, int t, int t_max,
                                float alpha, int32_t *assoc, int32_t *survivor,
                                void *cuda_stream) {
  if (m < 2 || m > kMaxM || n < 1 || r < 1 || !F || !V || !gamma || !assoc || !survivor ||
      t_max < 1 || !(alpha > 0.0f))
    return RVEA_ERR_ARG;
  // work items: every block of solutions x every chunk of vectors
  const int m4 = (m + 3) / 4;
  const SelPlan sp = sel_plan(n, r, m4, current_sm_count());
  const int nblk = sp.nblk, nch = sp.nch;
  const int n_items = nblk * nch;
  if (n > kNoAllocMaxN || r > kNoAllocMaxR) return RVEA_ERR_NOMEM;
  const Carve c = carve(n, r, m, n_items);
  if (c.total > kNoAllocBytes) return RVEA_ERR_NOMEM;

  unsigned char *ws = nullptr;
  const rvea_status s0 = scratch_for_current_device(&ws);
  if (s0 != RVEA_OK) return s0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  float *V32 = reinterpret_cast<float *>(ws + c.v32);
  RunDesc D;
  std::memset(&D, 0, sizeof(D));
  D.m = m; D.m4 = m4; D.N = r; D.n_comb = n; D.t_max = t_max; D.alpha = alpha;
  D.op_mode = 1; D.t_op = t;
  D.best = reinterpret_cast<unsigned long long *>(ws + c.best);
  D.amax = reinterpret_cast<unsigned long long *>(ws + c.amax);
  D.blk_cnt = reinterpret_cast<int *>(ws + c.blk);
  D.assoc = assoc;
  D.V32 = V32;
  D.gamma32 = const_cast<float *>(gamma);
  D.ctl = reinterpret_cast<Ctl *>(ws + c.ctl);
  D.F_aos = F;
  D.valid_in = valid;
  D.survivor_out = survivor;
  RunDesc *dD = reinterpret_cast<RunDesc *>(ws + c.desc);
  SelItem *items = reinterpret_cast<SelItem *>(ws + c.items);
  const int nset = std::max(n_items, r * 4 * m4);
  k_noalloc_setup<<<std::min(1024, (nset + 255) / 256), 256, 0, st>>>(D, dD, items, nblk, nch,
                                                                        sp.chunk, V, V32);
  // k_op_prep clears best, amax, the arrival counters and the control block
  k_op_prep<<<std::max(1, std::min(1024, (n + 255) / 256)), 256, 0, st>>>(dD);
  k_op_zstar<<<(n + 255) / 256, 256, 0, st>>>(dD);
  static thread_local BatchDir dir;
  dir.n = 1;
  dir.prefix[0] = 0;
  dir.prefix[1] = n_items;
  dir.desc[0] = dD;
  dir.items[0] = items;
  k_select<<<(unsigned)n_items, kSelThreads, std::min(r, sp.chunk) * m4 * 16, st>>>(dir);
  k_op_finish<<<(r + 255) / 256, 256, 0, st>>>(dD);
  return cudaGetLastError() == cudaSuccess ? RVEA_OK : RVEA_ERR_CUDA;
}

}  // extern "C"
