// jt_infer_device_noalloc: batched inference whose per-batch tables live in
// a fixed, file-scope device array instead of memory allocated by the plan.
//
// Some callers cannot allocate device memory at inference time: processes
// whose device memory is entirely reserved by another allocator (a
// framework's caching pool), serving loops that must not pay for
// cudaMalloc/cudaFree (they synchronise the device and stall every other
// stream), and deployments that forbid dynamic allocation after start-up.
// For them this entry point runs the same kernels as jt_infer_device with
// the arena carved out of g_jt_scratch.  It calls no cudaMalloc, cudaFree or
// other allocating routine; the plan (compiled earlier) is an input.
#include <mutex>

#include "kernels.cuh"
#include "runtime.h"

namespace {

constexpr size_t kScratchBytes = (size_t)JT_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_jt_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_jt_scratch on `device` (which must be current).  In
// host code the array's name is only a stand-in, so the address is looked up
// once per device and cached.
jt_status scratch_for(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) {
    jt::set_error("device ordinal out of range for the static scratch table");
    return JT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_jt_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      jt::set_error(std::string("cudaGetSymbolAddress(g_jt_scratch): ") + cudaGetErrorString(e));
      return JT_ECUDA;
    }
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return JT_OK;
}

}  // namespace

static jt_status jt_infer_device_noalloc_impl(jt_plan *pl, int32_t n_cases, const int32_t *d_ev,
                                             double *d_lp, double *d_post, int32_t *d_st,
                                             void *stream) {
  using namespace jt;
  if (!pl || n_cases < 0) { set_error("bad plan or n_cases"); return JT_EINVAL; }
  if (pl->host_only) { set_error("plan compiled with host_only"); return JT_EINVAL; }
  if (n_cases == 0) return JT_OK;
  if (!d_ev || !d_lp || !d_post || !d_st) { set_error("null buffer"); return JT_EINVAL; }
  const Plan &P = pl->P;
  const ArenaLayout L = arena_layout(P);
  if (L.bytes(1) > kScratchBytes) {
    set_error("this plan needs " + std::to_string(L.bytes(1)) + " bytes of scratch for one case tile; "
              "the static scratch holds " + std::to_string(kScratchBytes) + " bytes");
    return JT_ENOMEM;
  }
  if (cudaSetDevice(pl->device) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaSetDevice failed");
    return JT_ECUDA;
  }
  void *scratch = nullptr;
  jt_status st = scratch_for(pl->device, &scratch);
  if (st != JT_OK) return st;
  const int tiles =
      (int)std::min<size_t>((kScratchBytes - ArenaLayout::kTail) / L.per_tile, (size_t)kMaxTilesPerChunk);
  Arena a;
  st = arena_wrap(P, a, scratch, kScratchBytes, tiles);
  if (st != JT_OK) return st;
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : pl->stream;
  const int W = P.tile;
  const int64_t chunk = (int64_t)tiles * W;
  // the array keeps the previous call's contents: the split-sum counters
  // and the expired-wait flag must start at zero (so an expired wait of an
  // earlier call is not carried into this one; the other per-chunk state is
  // cleared by the passes themselves)
  if (cudaMemsetAsync(a.da.counters, 0, L.counters * (size_t)tiles, s) != cudaSuccess ||
      cudaMemsetAsync(a.da.errflag, 0, sizeof(uint32_t), s) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMemsetAsync on the static scratch failed");
    return JT_ECUDA;
  }
  for (int64_t b = 0; b < n_cases; b += chunk) {
    const int32_t nc = (int32_t)std::min<int64_t>(chunk, n_cases - b);
    DevArena A = a.da;
    A.tiles = (nc + W - 1) / W;
    cudaMemsetAsync(A.bad, 0, L.bad * (size_t)A.tiles, s);
    launch_evidence(P.cpt_per_thread, d_ev + b * P.io_n, nc, pl->dp, A, s);
    enqueue_passes(pl, A, s);
    launch_finalize(P.cpt_per_thread, pl->dp, A, nc, P.dcl[P.root].sep_row, d_lp + b, d_post + b * P.io_sum_card,
                    d_st + b, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("launch on the static scratch: ") + cudaGetErrorString(e));
    return JT_ECUDA;
  }
  return JT_OK;
}

extern "C" jt_status jt_infer_device_noalloc(jt_plan *pl, int32_t n_cases, const int32_t *d_ev,
                                             double *d_lp, double *d_post, int32_t *d_st,
                                             void *stream) {
  return jt::guarded([&] { return jt_infer_device_noalloc_impl(pl, n_cases, d_ev, d_lp, d_post, d_st, stream); });
}
