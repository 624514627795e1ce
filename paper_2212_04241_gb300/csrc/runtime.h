// Runtime objects behind the opaque jt_plan handle.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>

#include "kernels.cuh"

namespace jt {

// Bytes of one case tile in each arena region.
struct ArenaLayout {
  size_t psi, sep, post, partial, maxbits, counters, ev, bad, ready;
  size_t per_tile;
  // once per arena: the error flag (offset 0) and the dataflow unit
  // counters (offsets 64 and 192)
  static constexpr size_t kTail = 256;
  static constexpr size_t kQueueOffset = 64;
  size_t bytes(int tiles) const { return per_tile * (size_t)tiles + kTail; }
};

// Device memory for the per-batch tables of up to `tiles` case tiles, and
// the CUDA graphs captured against it (one per tile count).
struct Arena {
  void *mem = nullptr;
  size_t bytes = 0;        // bytes of the current layout
  size_t alloc_bytes = 0;  // bytes of the allocation (>= bytes)
  int tiles = 0;
  bool owns = true;
  DevArena da{};
  std::map<int, cudaGraphExec_t> graphs;
};

struct PlainWork {
  double *base = nullptr, *psi = nullptr, *sep = nullptr, *tmp = nullptr, *marg = nullptr, *pe = nullptr;
  int64_t *pool = nullptr, *post_off = nullptr;
  int32_t *card = nullptr, *ev = nullptr;
};

ArenaLayout arena_layout(const Plan &P);
jt_status arena_alloc(const Plan &P, Arena &a, int tiles);
jt_status arena_wrap(const Plan &P, Arena &a, void *mem, size_t bytes, int tiles);
void arena_free(Arena &a);

}  // namespace jt

struct jt_plan {
  jt::Plan P;
  bool host_only = false;
  int device = 0;
  cudaStream_t stream = nullptr;          // default stream of the plan
  cudaStream_t capture_stream = nullptr;  // private stream for graph capture
  void *d_static = nullptr;
  size_t static_bytes = 0;
  void *d_work = nullptr;                 // work lists (items, flow tables), replaced by retile
  size_t work_bytes = 0;
  int flow_collect_blocks = 0;            // dataflow grids: SMs x resident blocks per SM
  int flow_distribute_blocks = 0;
  jt::DevPlan dp{};
  jt::Arena arena;                        // default arena of jt_infer / jt_infer_device
  int budget_tiles_cache = 0;
  // staging for host-buffer calls
  void *d_io = nullptr, *h_io = nullptr;
  size_t io_ev = 0, io_lp = 0, io_post = 0, io_st = 0;
  int io_cases = 0;
  // plain FP64 path
  void *d_plain = nullptr;
  jt::PlainWork pw;
  std::mutex mu;
};

namespace jt {
// give a compiled plan the work shape of opts (items_per_tile*, rows_per_cta,
// *_rows_by_bucket): new work lists uploaded, graphs dropped, the arena
// rebound in place when the new layout fits it (else freed)
jt_status retile(jt_plan *pl, const jt_compile_opts &opts);
jt_status run_chunk(jt_plan *pl, Arena &a, const int32_t *d_ev, int32_t nc, double *d_lp, double *d_post,
                    int32_t *d_st, cudaStream_t s);
// JT_ETIMEOUT (and the flag cleared) when a kernel reported an expired
// bounded wait on this arena; call after synchronising its stream
jt_status check_arena_flag(Arena &a);
int budget_tiles(const jt_plan *pl, int64_t budget_bytes);
// the collect and distribute passes of one chunk (after its evidence
// kernel, before its finalize kernels), in the plan's schedule
void enqueue_passes(const jt_plan *pl, const DevArena &A, cudaStream_t s);
// the launch of one tree layer (layer schedule)
void enqueue_collect_layer(const jt_plan *pl, const DevArena &A, int layer, cudaStream_t s);
void enqueue_distribute_layer(const jt_plan *pl, const DevArena &A, int layer, cudaStream_t s);
}  // namespace jt
