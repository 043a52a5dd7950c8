// pspec_catalog_sums_noalloc: the catalog sums of pspec_paint (alpha, I, S and the sums
// they are built from) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA graph that is being
// captured, allocator-less embedded runtimes, or frameworks that hand every byte of the
// device to their own pool and forbid allocations behind their back. This entry point
// needs no workspace: its scratch (the per-block partial sums) lives in a file-scope
// __device__ array of fixed size that every GPU loading the library holds until exit.
#include <cuda_runtime.h>
#include <mutex>
#include "pspec.h"
#include "launch.h"

using namespace pspec;

namespace {

constexpr int kMaxDevices = 64;
// 2 catalogs x PSPEC_NOALLOC_MAX_BLOCKS partials x kSumVals doubles = 64 KiB.
constexpr int kScratchDoubles = 2 * PSPEC_NOALLOC_MAX_BLOCKS * kSumVals;

static __device__ __align__(256) double g_sums_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// The device address of g_sums_scratch on the current device. In host code the symbol is
// only a host-side stand-in, so the address is looked up once per device (the first call on a
// device, with that device current) and cached. cudaDeviceReset destroys the context the
// address belongs to: a process that resets a device must not call this entry point on it
// again.
pspec_status scratch_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PSPEC_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sums_scratch) != cudaSuccess || !p) return PSPEC_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return PSPEC_OK;
}

bool catalog_ok(const pspec_catalog* c, bool need_points) {
  if (!c || c->count < 0) return false;
  if (need_points && c->count == 0) return false;
  if (c->count > 0 && !c->pos) return false;
  return c->pos_dtype == PSPEC_POS_F64 || c->pos_dtype == PSPEC_POS_F32;
}

PaintArgs args_for(const pspec_params* p, const pspec_catalog* c) {
  PaintArgs a;
  a.pos = c->pos;
  a.pos_f32 = c->pos_dtype == PSPEC_POS_F32;
  a.weight = c->weight;
  a.nbar = c->nbar;
  a.count = c->count;
  for (int d = 0; d < 3; d++) a.corner[d] = p->box_corner[d];
  a.inv_cell = (double)p->nmesh / p->box_size;
  a.P0 = p->P0;
  a.nbar_default = p->nbar;
  a.wf_default = p->P0 > 0 ? 1.0 / (1.0 + p->nbar * p->P0) : 1.0;
  a.dc = nullptr;
  a.cur = nullptr;
  return a;
}

}  // namespace

extern "C" pspec_status pspec_catalog_sums_noalloc(const pspec_params* p, const pspec_catalog* data,
                                                   const pspec_catalog* randoms, int32_t nblocks, double* out,
                                                   void* stream) {
  if (!p || !out || !catalog_ok(data, false) || !catalog_ok(randoms, true)) return PSPEC_EINVAL;
  if (!(p->box_size > 0) || p->nmesh < 1) return PSPEC_EINVAL;
  if (nblocks < 0 || nblocks > PSPEC_NOALLOC_MAX_BLOCKS) return PSPEC_EINVAL;
  // An error already pending on this thread is the caller's: report it without launching and
  // leave it in place, so that the status below belongs to this call's launches alone.
  if (cudaPeekAtLastError() != cudaSuccess) return PSPEC_ECUDA;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PSPEC_ECUDA;
  if (nblocks == 0) nblocks = 2 * nsm < PSPEC_NOALLOC_MAX_BLOCKS ? 2 * nsm : PSPEC_NOALLOC_MAX_BLOCKS;
  double* scratch = nullptr;
  pspec_status st = scratch_on_current_device(&scratch);
  if (st != PSPEC_OK) return st;
  // Every partial the final sum reads is written by this call, so nothing needs clearing.
  double* part_d = scratch;
  double* part_r = scratch + (size_t)PSPEC_NOALLOC_MAX_BLOCKS * kSumVals;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  launch_catalog_partials(args_for(p, data), part_d, nblocks, s);
  if (cudaGetLastError() != cudaSuccess) return PSPEC_ECUDA;
  launch_catalog_partials(args_for(p, randoms), part_r, nblocks, s);
  if (cudaGetLastError() != cudaSuccess) return PSPEC_ECUDA;
  launch_catalog_final(part_d, nblocks, part_r, nblocks, out, s);
  return cudaGetLastError() == cudaSuccess ? PSPEC_OK : PSPEC_ECUDA;
}
