// Message kernels of the batched FP32 junction-tree path and of the plain
// FP64 comparator path.
//
// Batched path.  The unit of work is one warp's item (a row range of one
// clique's table, or of one distribute task) on one case tile.  Section 2
// packs all table entries of a BFS layer into one parallel task; here either
// one launch per layer and pass covers every item of the layer for every
// case tile (layer schedule: grid = item blocks x tiles), or one persistent
// launch per pass takes (item, tile) units in layer order and starts each
// as soon as its producers on the same tile are done (dataflow schedule).
// Tables are [tile][row][W] with W = 32 * CPT consecutive evidence cases per
// row; a warp moves one whole row (W * 4 bytes, fully coalesced) per access,
// so every index computation is shared by the W cases of a row.  Row indices
// are computed 32 rows at a time, one row per lane, and broadcast; rows are
// loaded four at a time (two at 8 cases per thread).
//
//   collect (Section 2: reduction + extension + marginalisation, fused):
//     psi_C[e] = base_C[e] * [evidence entered in C] *
//                prod_children phi*_child[map(e)] * 2^-k_child
//     phi*_C[s] = [evidence entered in S_up] * sum_u psi_C[s*R + u]
//                                              (upward separator outermost)
//     k_C = exponent of max_s phi*_C[s]          (power-of-two rescaling)
//   distribute (Hugin: extension by the separator ratio + marginalisation):
//     for every child separator and owned posterior variable T of C,
//     m_T[t] = sum_u psi_C[A[t]+B[u]] * rho_C[sA[t]+sB[u]]
//     rho_child = m_T / phi*_child  (0/0 := 0)
//   finalize: log P(e) = sum over component roots of ln(total) +
//     (sum of the other cliques' k + base exponents) ln 2, and the posterior
//     normalisation, both in FP64.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "kernels.cuh"

namespace jt {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// Rows whose loads a warp issues together, by kernel and cases per thread:
// a group holds 16 cases per lane at most, so wider tiles load fewer rows.
template <int CPT>
constexpr int kCollectGroup = CPT >= 8 ? 2 : 4;
template <int CPT>
constexpr int kDistGroup = CPT >= 8 ? 2 : 4;
// Resident blocks per SM the register allocation aims at: the collect
// kernel keeps its row group in registers without spilling at 2; the
// distribute kernel streams psi and gains from more warps in flight.
constexpr int kCollectBlocksPerSM = 2;
constexpr int kDistributeBlocksPerSM = 4;
// the distribute kernels of plans with fused pairs run both item kinds in
// one row loop, at the plain kernel's occupancy
constexpr int kFusedBlocksPerSM = 3;

// CPT cases of one thread inside a row of W = 32*CPT cases.  For CPT >= 4
// the thread holds CPT/4 float4 pieces, piece v at columns 128*v + 4*lane;
// for CPT < 4 one piece at columns CPT*lane.  Every access of a warp to a
// row is a contiguous 512-byte (or 128/256-byte) transaction per piece.
template <int CPT>
struct Vec {
  float x[CPT];
};

template <int CPT>
__device__ __forceinline__ int col_of(int lane, int k) {
  if constexpr (CPT >= 4) return 128 * (k >> 2) + 4 * lane + (k & 3);
  else return CPT * lane + k;
}

template <int CPT>
__device__ __forceinline__ Vec<CPT> vzero() {
  Vec<CPT> r;
#pragma unroll
  for (int k = 0; k < CPT; ++k) r.x[k] = 0.f;
  return r;
}

template <int CPT>
__device__ __forceinline__ Vec<CPT> vsplat(float a) {
  Vec<CPT> r;
#pragma unroll
  for (int k = 0; k < CPT; ++k) r.x[k] = a;
  return r;
}

enum LoadMode { LD_PLAIN, LD_STREAM, LD_NC, LD_CG };

template <LoadMode M, class T>
__device__ __forceinline__ T ld1(const T *p) {
  if constexpr (M == LD_STREAM) return __ldcs(p);
  else if constexpr (M == LD_NC) return __ldg(p);
  else if constexpr (M == LD_CG) return __ldcg(p);
  else return *p;
}

// Load this thread's CPT cases of the row starting at `row`.
template <int CPT, LoadMode M = LD_PLAIN>
__device__ __forceinline__ Vec<CPT> ldrow(const float *row, int lane) {
  Vec<CPT> r;
  if constexpr (CPT >= 4) {
#pragma unroll
    for (int v = 0; v < CPT / 4; ++v) {
      const float4 t = ld1<M>(reinterpret_cast<const float4 *>(row + 128 * v + 4 * lane));
      r.x[4 * v] = t.x; r.x[4 * v + 1] = t.y; r.x[4 * v + 2] = t.z; r.x[4 * v + 3] = t.w;
    }
  } else if constexpr (CPT == 2) {
    const float2 t = ld1<M>(reinterpret_cast<const float2 *>(row + 2 * lane));
    r.x[0] = t.x; r.x[1] = t.y;
  } else {
    r.x[0] = ld1<M>(row + lane);
  }
  return r;
}

template <int CPT, bool STREAM = false>
__device__ __forceinline__ void strow(float *row, int lane, const Vec<CPT> &a) {
  if constexpr (CPT >= 4) {
#pragma unroll
    for (int v = 0; v < CPT / 4; ++v) {
      float4 *p = reinterpret_cast<float4 *>(row + 128 * v + 4 * lane);
      const float4 t = make_float4(a.x[4 * v], a.x[4 * v + 1], a.x[4 * v + 2], a.x[4 * v + 3]);
      if constexpr (STREAM) __stcs(p, t); else *p = t;
    }
  } else if constexpr (CPT == 2) {
    float2 *p = reinterpret_cast<float2 *>(row + 2 * lane);
    const float2 t = make_float2(a.x[0], a.x[1]);
    if constexpr (STREAM) __stcs(p, t); else *p = t;
  } else {
    if constexpr (STREAM) __stcs(row + lane, a.x[0]); else row[lane] = a.x[0];
  }
}

// Paired FP32 arithmetic (Blackwell add/sub/mul .rn.f32x2): two cases per
// instruction, each element rounded exactly like the scalar operation.
__device__ __forceinline__ void mul2(float &a0, float &a1, float b0, float b1) {
  asm("{\n .reg .b64 pa, pb;\n mov.b64 pa, {%0, %1};\n mov.b64 pb, {%2, %3};\n"
      " mul.rn.f32x2 pa, pa, pb;\n mov.b64 {%0, %1}, pa;\n}"
      : "+f"(a0), "+f"(a1)
      : "f"(b0), "f"(b1));
}
__device__ __forceinline__ void add2(float &a0, float &a1, float b0, float b1) {
  asm("{\n .reg .b64 pa, pb;\n mov.b64 pa, {%0, %1};\n mov.b64 pb, {%2, %3};\n"
      " add.rn.f32x2 pa, pa, pb;\n mov.b64 {%0, %1}, pa;\n}"
      : "+f"(a0), "+f"(a1)
      : "f"(b0), "f"(b1));
}
__device__ __forceinline__ void sub2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
  asm("{\n .reg .b64 pa, pb;\n mov.b64 pa, {%2, %3};\n mov.b64 pb, {%4, %5};\n"
      " sub.rn.f32x2 pa, pa, pb;\n mov.b64 {%0, %1}, pa;\n}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// a *= b per case
template <int CPT>
__device__ __forceinline__ void vmul(Vec<CPT> &a, const Vec<CPT> &b) {
  if constexpr (CPT >= 2) {
#pragma unroll
    for (int k = 0; k < CPT; k += 2) mul2(a.x[k], a.x[k + 1], b.x[k], b.x[k + 1]);
  } else {
    a.x[0] *= b.x[0];
  }
}

// a += b per case
template <int CPT>
__device__ __forceinline__ void vadd(Vec<CPT> &a, const Vec<CPT> &b) {
  if constexpr (CPT >= 2) {
#pragma unroll
    for (int k = 0; k < CPT; k += 2) add2(a.x[k], a.x[k + 1], b.x[k], b.x[k + 1]);
  } else {
    a.x[0] += b.x[0];
  }
}

// Compensated (Kahan) accumulation per case of a partial sum: long FP32
// sums keep a few ulp.
template <int CPT>
__device__ __forceinline__ void kahan_fold(Vec<CPT> &sum, Vec<CPT> &comp, Vec<CPT> &part) {
  if constexpr (CPT >= 2) {
#pragma unroll
    for (int k = 0; k < CPT; k += 2) {
      float y0, y1, d0, d1;
      sub2(y0, y1, part.x[k], part.x[k + 1], comp.x[k], comp.x[k + 1]);  // y = part - comp
      float t0 = sum.x[k], t1 = sum.x[k + 1];
      add2(t0, t1, y0, y1);                                               // t = sum + y
      sub2(d0, d1, t0, t1, sum.x[k], sum.x[k + 1]);                       // t - sum
      sub2(comp.x[k], comp.x[k + 1], d0, d1, y0, y1);                     // comp = (t - sum) - y
      sum.x[k] = t0;
      sum.x[k + 1] = t1;
      part.x[k] = 0.f;
      part.x[k + 1] = 0.f;
    }
  } else {
    const float y = part.x[0] - comp.x[0];
    const float t = sum.x[0] + y;
    comp.x[0] = (t - sum.x[0]) - y;
    sum.x[0] = t;
    part.x[0] = 0.f;
  }
}

// Power-of-two exponent k of a non-negative float given by its bits, so
// that m * 2^-k lies in [1, 2) for normal m; 0 for m = 0, clamped to
// [-126, 126] so that 2^-k stays a normal float.
__device__ __forceinline__ int pow2_exp(uint32_t bits) {
  if (bits == 0) return 0;
  int e = (int)((bits >> 23) & 0xff);
  int k = (e == 0) ? -126 : e - 127;
  return max(-126, min(126, k));
}

// 2^k for k in [-126, 127], exact.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// ---------------------------------------------------------------------------
// evidence: [case][var] -> [tile][var][W], invalid states flagged
// ---------------------------------------------------------------------------
// A block moves 32 cases x 32 variables through shared memory, so both the
// [case][var] reads and the [tile][var][W] writes are coalesced.  Cases of
// the chunk's last tile beyond n_cases get -1 (unobserved).  Rows of
// ev_in have io_n columns (the full network of a pruned plan); the blocks
// past the kept variables check that the removed ones are unobserved.
__global__ void k_evidence(const int32_t *__restrict__ ev_in, int32_t n_cases, DevPlan P, DevArena A, int W) {
  __shared__ int32_t t[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int nvb = (P.n_vars + 31) / 32;
  if ((int)blockIdx.y >= nvb) {
    const int k = ((int)blockIdx.y - nvb) * 32 + threadIdx.x;
    if (k < P.n_dropped)
      for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i;
        if (c < n_cases && ev_in[c * P.io_n + P.io_dropped[k]] != -1) A.bad[c] = 1;
      }
    return;
  }
  const int v0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i;
    const int v = v0 + threadIdx.x;
    int val = -1;
    // a sliced plan's observed-set variables index the base tables: always a
    // valid state (0 stands in where a case breaks the contract or pads the tile)
    const bool in_set = P.slice_var != nullptr && v < P.n_vars && P.slice_var[v] != 0;
    if (v < P.n_vars && c < n_cases) {
      val = ev_in[c * P.io_n + (P.io_var ? P.io_var[v] : v)];
      if (val < -1 || val >= P.card[v] || (in_set && val < 0)) {
        A.bad[c] = 1;
        val = -1;
      }
    }
    if (in_set && val < 0) val = 0;
    t[i][threadIdx.x] = val;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int v = v0 + j;
    const int64_t c = c0 + threadIdx.x;
    if (v < P.n_vars && c < (int64_t)A.tiles * W) A.ev[((c / W) * P.n_vars + v) * W + (c % W)] = t[threadIdx.x][j];
  }
}

// ---------------------------------------------------------------------------
// shared pieces of the layer kernels
// ---------------------------------------------------------------------------
//
// The unit of work is one warp: an item (DItem) gives a warp whole segments
// of one table, or a row range of one segment ("split" item).  A block holds
// kWarps independent items -- possibly of different cliques -- and never
// synchronises, so small cliques pack together and no warp waits for another.

// Rows of a warp's item: non-split items own whole segments [t0, t0+nt) of
// R rows each (flattened in segment order); split items own rows
// [u0, u0+nu) of segment t0.
__device__ __forceinline__ void item_rows(const DItem &it, int32_t R, int32_t &s_first, int32_t &u_first,
                                          int32_t &count) {
  s_first = (int32_t)it.t0;
  if (!it.split) {
    u_first = 0;
    count = (int32_t)(it.nt * (int64_t)R);
  } else {
    u_first = (int32_t)it.u0;
    count = (int32_t)it.nu;
  }
}

// Combine the partial sums of a split segment: every piece (one warp) writes
// its sum, and the last piece to finish adds all of them in piece order.
// Returns true in the warp that holds the final value, with `tot` set.
template <int CPT>
__device__ __forceinline__ bool combine_split(const DItem &it, const DevPlan &P, const DevArena &A, int tile,
                                              int lane, const Vec<CPT> &acc, Vec<CPT> &tot) {
  constexpr int W = 32 * CPT;
  if (it.npieces == 1) {
    tot = acc;
    return true;
  }
  strow<CPT>(A.partial + ((int64_t)tile * P.n_partials + it.partial) * W, lane, acc);
  __threadfence();
  __syncwarp();
  unsigned old = 0;
  if (lane == 0) old = atomicAdd(&A.counters[(int64_t)tile * P.n_groups + it.group], 1u);
  old = __shfl_sync(kFull, old, 0);
  if (old != (unsigned)(it.npieces - 1)) return false;
  __threadfence();
  const int first = it.partial - it.piece;
  tot = vzero<CPT>();
  for (int p = 0; p < it.npieces; ++p) {
    const Vec<CPT> x = ldrow<CPT, LD_CG>(A.partial + ((int64_t)tile * P.n_partials + first + p) * W, lane);
#pragma unroll
    for (int k = 0; k < CPT; ++k) tot.x[k] += x.x[k];
  }
  if (lane == 0) A.counters[(int64_t)tile * P.n_groups + it.group] = 0u;
  return true;
}

// ---------------------------------------------------------------------------
// collect
// ---------------------------------------------------------------------------

// Shared memory of one warp: per map (child and evidence maps, then the
// evidence of the upward message) its per-case value -- the child message's
// scale 2^-k, or the observed state (-1 if unobserved) -- read as float4, so
// it comes first and every part is rounded to 16 bytes; its index-table
// offsets and message row; and the map indices of 32 rows.
__host__ __device__ inline size_t round16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline size_t collect_warp_smem(int cpt, int nm) {
  const int W = 32 * cpt;
  return round16(sizeof(float) * W * (size_t)nm) + round16(3 * sizeof(int64_t) * (size_t)nm) +
         round16(sizeof(int32_t) * 32 * (size_t)nm);
}

// Per-warp shared memory of a clique's maps (the layout collect_warp_smem
// sizes): per map its per-case value, its index-table offsets and message
// row, and the map indices of 32 rows.
template <int CPT>
struct MapSmem {
  float *mval;
  int64_t *mA, *mB, *mrow;
  int32_t *idx;
  __device__ __forceinline__ MapSmem(unsigned char *ws, int max_maps) {
    constexpr int W = 32 * CPT;
    mval = reinterpret_cast<float *>(ws);
    mA = reinterpret_cast<int64_t *>(ws + round16(sizeof(float) * W * (size_t)max_maps));
    mB = mA + max_maps;
    mrow = mB + max_maps;
    idx = reinterpret_cast<int32_t *>(ws + round16(sizeof(float) * W * (size_t)max_maps) +
                                      round16(3 * sizeof(int64_t) * (size_t)max_maps));
  }
};

// Load clique C's maps [map_begin, map_begin + nmaps) into the warp's shared
// memory.  Child maps gather rows of the child's message (scaled by 2^-k
// per case); evidence maps keep each case's observed state: an entry whose
// digit of the variable differs from it is zeroed (the 0/1 indicator of the
// reduction step, evaluated instead of loaded).  Child maps come first.
// Returns the number of child maps.
template <int CPT>
__device__ __forceinline__ int load_clique_maps(const DevPlan &P, const DevArena &A, const DClique &C, int nmaps,
                                                int tile, const MapSmem<CPT> &sm, int lane) {
  constexpr int W = 32 * CPT;
  int nchild = 0;
  for (int i = 0; i < nmaps; ++i) {
    const DMap mp = P.maps[C.map_begin + i];
    const bool child = mp.kind == MAP_CHILD;
    if (lane == 0) {
      sm.mA[i] = mp.A_off;
      sm.mB[i] = mp.B_off;
      sm.mrow[i] = child ? (A.phistar - A.psi) + ((int64_t)tile * P.sep_rows + mp.src_row) * W : 0;
    }
    nchild += child;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      const int c = col_of<CPT>(lane, k);
      sm.mval[i * W + c] = child ? (P.rescale ? pow2f(-pow2_exp(A.maxbits[((int64_t)tile * P.n_cliques + mp.src) * W + c]))
                                              : 1.f)
                                 : (float)A.ev[((int64_t)tile * P.n_vars + mp.src) * W + c];
    }
  }
  __syncwarp();
  return nchild;
}

// The clique table's rows r .. r+G-1 of a 32-row batch, per case: the base
// entry (lane j holds row j's; a sliced plan gathers each case's slice
// through fj and boff), times every child message row (gathered through the
// batch's map indices, scaled by 2^-k), zeroed where an evidence map's
// digit differs from the case's state -- the collect pass's reduction and
// extension, in one fixed order (so a recomputed row equals the stored one
// bit for bit).
template <int CPT, int G, LoadMode MSG, bool SLICED>
__device__ __forceinline__ void clique_rows(const DevArena &A, const MapSmem<CPT> &sm, const float *__restrict__ base,
                                            const int32_t (&boff)[CPT], bool sliced, float bj, int32_t fj, int nchild,
                                            int nm, int r, int nb, int lane, Vec<CPT> (&v)[G]) {
  constexpr int W = 32 * CPT;
  if (!sliced) {
#pragma unroll
    for (int g = 0; g < G; ++g) v[g] = vsplat<CPT>(__shfl_sync(kFull, bj, min(r + g, nb - 1)));
  } else {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int32_t f = __shfl_sync(kFull, fj, min(r + g, nb - 1));
#pragma unroll
      for (int k = 0; k < CPT; ++k) v[g].x[k] = __ldg(base + f + boff[k]);
    }
  }
  // child maps two at a time: both rows are requested before either is used
  for (int i = 0; i < nchild; i += 2) {
    const bool two = i + 1 < nchild;
    const float *mp0 = A.psi + sm.mrow[i];
    const float *mp1 = A.psi + sm.mrow[two ? i + 1 : i];
    Vec<CPT> m0[G], m1[G];
#pragma unroll
    for (int g = 0; g < G; ++g) m0[g] = ldrow<CPT, MSG>(mp0 + (int64_t)sm.idx[i * 32 + min(r + g, nb - 1)] * W, lane);
    if (two) {
#pragma unroll
      for (int g = 0; g < G; ++g)
        m1[g] = ldrow<CPT, MSG>(mp1 + (int64_t)sm.idx[(i + 1) * 32 + min(r + g, nb - 1)] * W, lane);
    }
    {
      const Vec<CPT> sc = ldrow<CPT>(sm.mval + i * W, lane);
#pragma unroll
      for (int g = 0; g < G; ++g) vmul<CPT>(m0[g], sc);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) vmul<CPT>(v[g], m0[g]);
    if (two) {
      {
        const Vec<CPT> sc = ldrow<CPT>(sm.mval + (i + 1) * W, lane);
#pragma unroll
        for (int g = 0; g < G; ++g) vmul<CPT>(m1[g], sc);
      }
#pragma unroll
      for (int g = 0; g < G; ++g) vmul<CPT>(v[g], m1[g]);
    }
  }
  for (int i = nchild; i < nm; ++i) {  // evidence maps: idx is the variable's digit
    const Vec<CPT> e = ldrow<CPT>(sm.mval + i * W, lane);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const float d = (float)sm.idx[i * 32 + min(r + g, nb - 1)];
#pragma unroll
      for (int k = 0; k < CPT; ++k) v[g].x[k] = (e.x[k] < 0.f || e.x[k] == d) ? v[g].x[k] : 0.f;
    }
  }
}

// One collect work item (a warp's rows of one clique, one case tile).  MSG
// is the load path of the children's messages: the read-only path when an
// earlier kernel wrote them, coherent loads when warps of the same kernel
// did (dataflow schedule).  SLICED instantiates the base-table gather of
// plans specialised to an observed set; other plans compile without it.
// A plan whose distribute pass recomputes the clique tables stores none.
template <int CPT, LoadMode MSG, bool SLICED>
__device__ __forceinline__ void collect_item(const DevPlan &P, const DevArena &A, const DItem &it, int tile,
                                             unsigned char *ws, int max_maps, int lane) {
  constexpr int W = 32 * CPT;
  constexpr int G = kCollectGroup<CPT>;
  const DClique C = P.cl[it.task];
  const int nm = C.map_end - C.map_begin;
  const MapSmem<CPT> sm(ws, max_maps);
  // the upward message's evidence maps follow the clique's maps
  const int nsev = C.sev_end - C.sev_begin;
  const int nchild = load_clique_maps<CPT>(P, A, C, nm + nsev, tile, sm, lane);
  const int32_t R = (int32_t)C.R;
  const float *__restrict__ base = P.base32 + C.base_off;
  // sliced plan: each case reads the base-table slice of its observed-set
  // states (offset in the full base table), entry e of the sliced table
  // being base entry bA[s] + bB[u]
  const bool sliced = SLICED && C.slice_end > C.slice_begin;
  int32_t boff[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) boff[k] = 0;
  for (int i = C.slice_begin; SLICED && i < C.slice_end; ++i) {
    const DMap mp = P.maps[i];
#pragma unroll
    for (int k = 0; k < CPT; ++k)
      boff[k] += A.ev[((int64_t)tile * P.n_vars + mp.src) * W + col_of<CPT>(lane, k)] * (int32_t)mp.A_off;
  }
  const int32_t *__restrict__ bA = P.ipool + C.bmap_A;
  const int32_t *__restrict__ bB = P.ipool + C.bmap_B;
  float *psi = A.psi + ((int64_t)tile * P.psi_rows + C.psi_row) * W;
  float *phi_out = A.phistar + ((int64_t)tile * P.sep_rows + C.sep_row) * W;
  const bool store = !P.recompute;

  // evidence entered into the upward message: entry s is zeroed for the
  // cases whose observed state of the variable differs from its digit at s
  auto sep_evidence = [&](int64_t s, Vec<CPT> &val) {
    for (int j = nm; j < nm + nsev; ++j) {
      const float d = (float)__ldg(P.ipool + sm.mA[j] + s);
      const Vec<CPT> e = ldrow<CPT>(sm.mval + j * W, lane);
#pragma unroll
      for (int k = 0; k < CPT; ++k) val.x[k] = (e.x[k] < 0.f || e.x[k] == d) ? val.x[k] : 0.f;
    }
  };

  int32_t s_first, u_first, count;
  item_rows(it, R, s_first, u_first, count);
  const int64_t e_first = (int64_t)s_first * R + u_first;  // rows are entries e_first + [0, count)
  Vec<CPT> mx = vzero<CPT>(), acc = vzero<CPT>(), comp = vzero<CPT>(), part = vzero<CPT>();
  for (int32_t b0 = 0; b0 < count; b0 += 32) {
    const int nb = min(32, count - b0);
    // lane j: indices of row b0 + j
    const int64_t ej = e_first + b0 + min(lane, nb - 1);
    const int32_t sj = (int32_t)ej / R, uj = (int32_t)ej - sj * R;  // |C| < 2^31
    const int32_t fj = sliced ? __ldg(bA + sj) + __ldg(bB + uj) : 0;  // base entry (sliced plan)
    const float bj = sliced ? 0.f : __ldg(base + ej);
    for (int i = 0; i < nm; ++i) sm.idx[i * 32 + lane] = __ldg(P.ipool + sm.mA[i] + sj) + __ldg(P.ipool + sm.mB[i] + uj);
    const unsigned last = __ballot_sync(kFull, !it.split && uj == R - 1 && lane < nb);
    __syncwarp();
    // collect_prefetch: the batch's child-message rows are requested into L2
    // at once (lane j: row j's), so every group's gathers find them there
    if (P.msg_prefetch != 0 && lane < nb) {
      for (int i = 0; i < nchild; ++i) {
        const float *pr = A.psi + sm.mrow[i] + (int64_t)sm.idx[i * 32 + lane] * W;
#pragma unroll
        for (int l = 0; l < W / 32; ++l) asm volatile("prefetch.global.L2 [%0];" ::"l"(pr + 32 * l));
      }
    }
    for (int r = 0; r < nb; r += G) {
      Vec<CPT> v[G];
      clique_rows<CPT, G, MSG, SLICED>(A, sm, base, boff, sliced, bj, fj, nchild, nm, r, nb, lane, v);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (r + g < nb) {
          if (store) strow<CPT, true>(psi + (e_first + b0 + r + g) * W, lane, v[g]);
          vadd<CPT>(part, v[g]);
          if ((last >> (r + g)) & 1u) {  // segment complete
            kahan_fold<CPT>(acc, comp, part);
            const int32_t s = __shfl_sync(kFull, sj, r + g);
            sep_evidence(s, acc);
            strow<CPT>(phi_out + (int64_t)s * W, lane, acc);
#pragma unroll
            for (int k = 0; k < CPT; ++k) mx.x[k] = fmaxf(mx.x[k], acc.x[k]);
            acc = vzero<CPT>();
            comp = vzero<CPT>();
          }
        }
      }
      kahan_fold<CPT>(acc, comp, part);
    }
    __syncwarp();
  }
  if (it.split) {
    Vec<CPT> tot;
    if (combine_split<CPT>(it, P, A, tile, lane, acc, tot)) {
      sep_evidence(it.t0, tot);
      strow<CPT>(phi_out + it.t0 * W, lane, tot);
#pragma unroll
      for (int k = 0; k < CPT; ++k) mx.x[k] = fmaxf(mx.x[k], tot.x[k]);
    }
  }
  // per-case maximum of the message entries this warp completed
  unsigned *mb = A.maxbits + ((int64_t)tile * P.n_cliques + it.task) * W;
#pragma unroll
  for (int k = 0; k < CPT; ++k)
    if (P.rescale && mx.x[k] > 0.f) atomicMax(mb + col_of<CPT>(lane, k), __float_as_uint(mx.x[k]));
}

template <int CPT, bool SLICED>
__global__ void __launch_bounds__(kThreads, kCollectBlocksPerSM) k_collect(DevPlan P, DevArena A, int64_t item_begin,
                                                          int64_t n_items, int max_maps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t iw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (iw >= n_items) return;
  collect_item<CPT, LD_NC, SLICED>(P, A, P.citems[item_begin + iw], blockIdx.y,
                                   smem_raw + (size_t)warp * collect_warp_smem(CPT, max_maps), max_maps, lane);
}

// ---------------------------------------------------------------------------
// distribute
// ---------------------------------------------------------------------------
// One distribute work item (a warp's rows of one task, one case tile).  RHO
// is the load path of the clique's ratio rows (see collect_item).
// RECOMP: the plan stores no clique tables; a task reading the clique's
// table recomputes each row it needs (clique_rows: the collect pass's
// product, in its order) from the base table, the child messages and the
// evidence, using the warp's shared memory `ws` for the clique's maps.
template <int CPT, LoadMode RHO, bool RECOMP = false>
__device__ __forceinline__ void distribute_item(const DevPlan &P, const DevArena &A, const DItem &it, int tile,
                                                int lane, unsigned char *ws = nullptr) {
  constexpr int W = 32 * CPT;
  constexpr int G = RECOMP ? kCollectGroup<CPT> : kDistGroup<CPT>;
  const DTask &T = P.tasks[it.task];
  const DClique &C = P.cl[T.clique];
  const bool recomp = RECOMP && !T.src_sep;  // a separator's phi* rows are stored
  MapSmem<CPT> sm(ws, RECOMP ? P.max_maps : 0);
  const int nm = C.map_end - C.map_begin;
  const int nchild = recomp ? load_clique_maps<CPT>(P, A, C, nm, tile, sm, lane) : 0;
  const float *__restrict__ base = P.base32 + C.base_off;
  const int32_t Rc = (int32_t)C.R;
  int32_t no_off[CPT];
#pragma unroll
  for (int k = 0; k < CPT; ++k) no_off[k] = 0;
  // X rows: the clique's psi, or the phi* rows of its upward separator
  const float *psi = T.src_sep ? A.phistar + ((int64_t)tile * P.sep_rows + C.sep_row) * W
                               : A.psi + ((int64_t)tile * P.psi_rows + C.psi_row) * W;
  const float *rho = A.rho + ((int64_t)tile * P.sep_rows + C.sep_row) * W;
  const bool root = !T.src_sep && C.is_root != 0;
  // a component root's scale 2^-k per case (computed where it is used, so
  // that it holds no registers through the row loop)
  auto root_scale = [&]() {
    Vec<CPT> rs;
#pragma unroll
    for (int k = 0; k < CPT; ++k)
      rs.x[k] = P.rescale ? pow2f(-pow2_exp(A.maxbits[((int64_t)tile * P.n_cliques + T.clique) * W + col_of<CPT>(lane, k)]))
                          : 1.f;
    return rs;
  };
  const int32_t U = (int32_t)T.U;

  auto output = [&](int64_t t, const Vec<CPT> &val) {
    if (T.kind == TASK_CHILD) {
      const int64_t o = ((int64_t)tile * P.sep_rows + T.dst_row + t) * W;
      const Vec<CPT> ph = ldrow<CPT>(A.phistar + o, lane);
      Vec<CPT> q;
#pragma unroll
      for (int k = 0; k < CPT; ++k) q.x[k] = (ph.x[k] > 0.f) ? val.x[k] / ph.x[k] : 0.f;  // 0/0 := 0
      strow<CPT>(A.rho + o, lane, q);
    } else {
      strow<CPT>(A.post + ((int64_t)tile * P.post_rows + T.dst_row + t) * W, lane, val);
    }
  };

  int32_t t_first, u_first, count;
  item_rows(it, U, t_first, u_first, count);
  Vec<CPT> acc = vzero<CPT>(), comp = vzero<CPT>(), part = vzero<CPT>();
  for (int32_t b0 = 0; b0 < count; b0 += 32) {
    const int nb = min(32, count - b0);
    // lane j: indices of row b0 + j, rows flattened as (t, u)
    const int32_t f = u_first + b0 + min(lane, nb - 1);
    const int32_t tj = t_first + f / U, uj = f - (f / U) * U;
    // the index tables are read through the task (no pointers held across
    // the row loop)
    const int32_t ej = __ldg(P.ipool + T.A_off + tj) + __ldg(P.ipool + T.B_off + uj);
    const int32_t xj = root ? 0 : __ldg(P.ipool + T.sA_off + tj) + __ldg(P.ipool + T.sB_off + uj);
    const unsigned last = __ballot_sync(kFull, !it.split && uj == U - 1 && lane < nb);
    float bj = 0.f;
    if (recomp) {  // lane j: the base entry and map indices of its row's clique entry
      const int32_t sj = ej / Rc, u2 = ej - sj * Rc;
      bj = __ldg(base + ej);
      for (int i = 0; i < nm; ++i) sm.idx[i * 32 + lane] = __ldg(P.ipool + sm.mA[i] + sj) + __ldg(P.ipool + sm.mB[i] + u2);
      __syncwarp();
    }
    for (int r = 0; r < nb; r += G) {
      Vec<CPT> p[G];
      if (recomp) {
        clique_rows<CPT, G, LD_NC, false>(A, sm, base, no_off, false, bj, 0, nchild, nm, r, nb, lane, p);
      } else {
#pragma unroll
        for (int g = 0; g < G; ++g)
          p[g] = ldrow<CPT, LD_STREAM>(psi + (int64_t)__shfl_sync(kFull, ej, min(r + g, nb - 1)) * W, lane);
      }
      // the next group's rows are requested into L2 now: more bytes in
      // flight at the register-limited occupancy, without holding registers
      if (!recomp && r + G < nb) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const float *pa = psi + (int64_t)__shfl_sync(kFull, ej, min(r + G + g, nb - 1)) * W + lane * CPT;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
        }
      }
      if (!root) {
        Vec<CPT> q[G];
#pragma unroll
        for (int g = 0; g < G; ++g)
          q[g] = ldrow<CPT, RHO>(rho + (int64_t)__shfl_sync(kFull, xj, min(r + g, nb - 1)) * W, lane);
#pragma unroll
        for (int g = 0; g < G; ++g) vmul<CPT>(p[g], q[g]);
      } else {
        const Vec<CPT> rs = root_scale();
#pragma unroll
        for (int g = 0; g < G; ++g) vmul<CPT>(p[g], rs);
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (r + g < nb) {
          vadd<CPT>(part, p[g]);
          if ((last >> (r + g)) & 1u) {  // target entry complete
            kahan_fold<CPT>(acc, comp, part);
            output(__shfl_sync(kFull, tj, r + g), acc);
            acc = vzero<CPT>();
            comp = vzero<CPT>();
          }
        }
      }
      kahan_fold<CPT>(acc, comp, part);
    }
    if (recomp) __syncwarp();  // the next batch rewrites the map indices
  }
  if (it.split) {
    Vec<CPT> tot;
    if (combine_split<CPT>(it, P, A, tile, lane, acc, tot)) output(it.t0, tot);
  }
}

// The work item of a plan with fused pairs: a single task's item (as
// distribute_item), or a fused pair's item (see DTask): whole primary
// targets [t0, t0 + nt) of one F-block, or whole F-blocks.  Both kinds run
// the same row loop.  In a fused item every row is read once: the primary
// target's sum runs in registers, the secondary targets of the F-block are
// summed in this warp's shared memory (sec_b rows of W floats, each lane
// its own CPT columns, so no two lanes touch the same word).  The 32-row
// batches of a fused item restart at every F-block, so an F-block ends with
// a batch and its secondary targets are written between batches, outside
// the loop that holds the rows in flight; a piece of an F-block writes its
// secondary sums as partials that the last piece to finish adds in piece
// order.
template <int CPT, LoadMode RHO>
__device__ __forceinline__ void distribute_pair_item(const DevPlan &P, const DevArena &A, const DItem &it, int tile,
                                                     int lane, float *sec) {
  constexpr int W = 32 * CPT;
  constexpr int G = kDistGroup<CPT>;
  const DTask &T = P.tasks[it.task];
  const DClique &C = P.cl[T.clique];
  const bool fz = it.fused != 0;
  const float *psi = T.src_sep ? A.phistar + ((int64_t)tile * P.sep_rows + C.sep_row) * W
                               : A.psi + ((int64_t)tile * P.psi_rows + C.psi_row) * W;
  const float *rho = A.rho + ((int64_t)tile * P.sep_rows + C.sep_row) * W;
  const bool root = !T.src_sep && C.is_root != 0;
  // a component root's scale 2^-k per case (computed where it is used, so
  // that it holds no registers through the row loop)
  auto root_scale = [&]() {
    Vec<CPT> rs;
#pragma unroll
    for (int k = 0; k < CPT; ++k)
      rs.x[k] = P.rescale ? pow2f(-pow2_exp(A.maxbits[((int64_t)tile * P.n_cliques + T.clique) * W + col_of<CPT>(lane, k)]))
                          : 1.f;
    return rs;
  };
  const int32_t U = (int32_t)T.U;
  const int32_t a = fz ? T.sec_a : 1, nb2 = fz ? T.sec_b : 0;

  // a target's value: a separator ratio (0/0 := 0) or a posterior marginal
  auto write = [&](int kind, int64_t row, const Vec<CPT> &val) {
    if (kind == TASK_CHILD) {
      const int64_t o = ((int64_t)tile * P.sep_rows + row) * W;
      const Vec<CPT> ph = ldrow<CPT>(A.phistar + o, lane);
      Vec<CPT> q;
#pragma unroll
      for (int k = 0; k < CPT; ++k) q.x[k] = (ph.x[k] > 0.f) ? val.x[k] / ph.x[k] : 0.f;
      strow<CPT>(A.rho + o, lane, q);
    } else {
      strow<CPT>(A.post + ((int64_t)tile * P.post_rows + row) * W, lane, val);
    }
  };
  // the primary target t's row (a fused pair's targets are enumerated in
  // F-block order, OP maps them back to the task's own rows)
  auto out_row = [&](int64_t t) -> int64_t {
    const DTask &Tt = P.tasks[it.task];
    return Tt.dst_row + (fz ? (int64_t)__ldg(P.ipool + Tt.op_off + t) : t);
  };
  auto sec_row = [&](int64_t f, int k) {
    const DTask &Tt = P.tasks[it.task];
    return Tt.sec_dst_row + __ldg(P.ipool + Tt.osf_off + f) + __ldg(P.ipool + Tt.osk_off + k);
  };
  // the secondary targets of F-block fb from shared memory (zeroed for the
  // next F-block); a separator ratio needs phi*, so the divisors of two
  // targets are requested together
  auto flush_sec = [&](int64_t fb) {
    const DTask &Tt = P.tasks[it.task];
    for (int k0 = 0; k0 < nb2; k0 += 2) {
      const int nk = min(2, nb2 - k0);
      int64_t row[2];
      Vec<CPT> val[2], ph[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        row[j] = j < nk ? sec_row(fb, k0 + j) : 0;
        val[j] = ldrow<CPT>(sec + (int64_t)(k0 + min(j, nk - 1)) * W, lane);
        if (Tt.sec_kind == TASK_CHILD && j < nk) ph[j] = ldrow<CPT>(A.phistar + ((int64_t)tile * P.sep_rows + row[j]) * W, lane);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (j >= nk) break;
        if (Tt.sec_kind == TASK_CHILD) {
          Vec<CPT> q;
#pragma unroll
          for (int c = 0; c < CPT; ++c) q.x[c] = (ph[j].x[c] > 0.f) ? val[j].x[c] / ph[j].x[c] : 0.f;  // 0/0 := 0
          strow<CPT>(A.rho + ((int64_t)tile * P.sep_rows + row[j]) * W, lane, q);
        } else {
          strow<CPT>(A.post + ((int64_t)tile * P.post_rows + row[j]) * W, lane, val[j]);
        }
        strow<CPT>(sec + (int64_t)(k0 + j) * W, lane, vzero<CPT>());
      }
    }
  };
  // the divisor rows (phi*) of an F-block's secondary targets are requested
  // into L2 when the F-block starts, so that its flush finds them there
  auto prefetch_sec = [&](int64_t fb) {
    const DTask &Tt = P.tasks[it.task];
    if (Tt.sec_kind != TASK_CHILD) return;
    constexpr int kLines = W * 4 / 128;  // 128-byte lines per row
    for (int j = lane; j < nb2 * kLines; j += 32) {
      const float *pa = A.phistar + ((int64_t)tile * P.sep_rows + sec_row(fb, j / kLines)) * W + (j % kLines) * 32;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
    }
  };

  int32_t t_first, u_first, count;
  item_rows(it, U, t_first, u_first, count);
  // relative row at which the next F-block ends (a fused item's batches
  // stop there); the rows of an F-block are a * U consecutive rows
  int32_t fb_next = fz ? (int32_t)((t_first / a + 1) * a - t_first) * U : 0x7fffffff;
  if (fz) {
    for (int k = 0; k < nb2; ++k) strow<CPT>(sec + (int64_t)k * W, lane, vzero<CPT>());
    prefetch_sec(t_first / a);
  }
  Vec<CPT> acc = vzero<CPT>(), comp = vzero<CPT>(), part = vzero<CPT>();
  for (int32_t b0 = 0; b0 < count;) {
    const int nb = min(min(32, count - b0), fb_next - b0);
    // lane j: indices of row b0 + j, rows flattened as (t, u)
    const int32_t f = u_first + b0 + min(lane, nb - 1);
    const int32_t tj = t_first + f / U, uj = f - (f / U) * U;
    const int32_t ej = __ldg(P.ipool + (fz ? T.fA_off : T.A_off) + tj) + __ldg(P.ipool + (fz ? T.fB_off : T.B_off) + uj);
    const int32_t xj =
        root ? 0 : __ldg(P.ipool + (fz ? T.fsA_off : T.sA_off) + tj) + __ldg(P.ipool + (fz ? T.fsB_off : T.sB_off) + uj);
    const int32_t kj = fz ? __ldg(P.ipool + T.ku_off + uj) : 0;
    const unsigned last = __ballot_sync(kFull, !it.split && uj == U - 1 && lane < nb);
    for (int r = 0; r < nb; r += G) {
      Vec<CPT> p[G];
#pragma unroll
      for (int g = 0; g < G; ++g)
        p[g] = ldrow<CPT, LD_STREAM>(psi + (int64_t)__shfl_sync(kFull, ej, min(r + g, nb - 1)) * W, lane);
      // the next group's rows are requested into L2 now: more bytes in
      // flight at the register-limited occupancy, without holding registers
      if (r + G < nb) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const float *pa = psi + (int64_t)__shfl_sync(kFull, ej, min(r + G + g, nb - 1)) * W + lane * CPT;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
        }
      }
      if (!root) {
        Vec<CPT> q[G];
#pragma unroll
        for (int g = 0; g < G; ++g)
          q[g] = ldrow<CPT, RHO>(rho + (int64_t)__shfl_sync(kFull, xj, min(r + g, nb - 1)) * W, lane);
#pragma unroll
        for (int g = 0; g < G; ++g) vmul<CPT>(p[g], q[g]);
      } else {
        const Vec<CPT> rs = root_scale();
#pragma unroll
        for (int g = 0; g < G; ++g) vmul<CPT>(p[g], rs);
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if (r + g < nb) {
          if (fz) {  // the secondary target of this row, summed in shared memory
            float *srow = sec + (int64_t)__shfl_sync(kFull, kj, r + g) * W;
            Vec<CPT> sv = ldrow<CPT>(srow, lane);
            vadd<CPT>(sv, p[g]);
            strow<CPT>(srow, lane, sv);
          }
          vadd<CPT>(part, p[g]);
          if ((last >> (r + g)) & 1u) {  // primary target complete
            kahan_fold<CPT>(acc, comp, part);
            write(P.tasks[it.task].kind, out_row(__shfl_sync(kFull, tj, r + g)), acc);
            acc = vzero<CPT>();
            comp = vzero<CPT>();
          }
        }
      }
      kahan_fold<CPT>(acc, comp, part);
    }
    b0 += nb;
    if (b0 == fb_next) {  // an F-block ended with this batch
      if (it.npieces == 1) {  // a whole F-block: its secondary targets
        const int64_t fb = (int64_t)(t_first + (b0 - 1) / U) / a;
        flush_sec(fb);
        if (b0 < count) prefetch_sec(fb + 1);
      }
      // whole F-blocks: the next one ends inside the item (no overflow)
      if (b0 < count) fb_next += a * U;
    }
  }
  if (it.split) {
    Vec<CPT> tot;
    if (combine_split<CPT>(it, P, A, tile, lane, acc, tot)) write(P.tasks[it.task].kind, out_row(it.t0), tot);
  }
  if (fz && it.npieces > 1) {
    // a piece of an F-block: partial secondary sums, combined in piece order
    // by the last piece to finish
    float *pbase = A.partial + ((int64_t)tile * P.n_partials + it.partial) * W;
    for (int k = 0; k < nb2; ++k) strow<CPT>(pbase + (int64_t)k * W, lane, ldrow<CPT>(sec + (int64_t)k * W, lane));
    __threadfence();
    __syncwarp();
    unsigned old = 0;
    if (lane == 0) old = atomicAdd(&A.counters[(int64_t)tile * P.n_groups + it.group], 1u);
    old = __shfl_sync(kFull, old, 0);
    if (old == (unsigned)(it.npieces - 1)) {
      __threadfence();
      const int64_t fb = it.t0 / a;
      const int first = it.partial - it.piece * nb2;
      // sum in piece order into the shared-memory rows (the loads of one
      // piece's rows are independent and issued together), then write the
      // targets as an F-block flush does
      for (int q = 0; q < it.npieces; ++q) {
#pragma unroll 4
        for (int k = 0; k < nb2; ++k) {
          const Vec<CPT> x =
              ldrow<CPT, LD_CG>(A.partial + ((int64_t)tile * P.n_partials + first + q * nb2 + k) * W, lane);
          Vec<CPT> t = q == 0 ? vzero<CPT>() : ldrow<CPT>(sec + (int64_t)k * W, lane);
#pragma unroll
          for (int c = 0; c < CPT; ++c) t.x[c] += x.x[c];
          strow<CPT>(sec + (int64_t)k * W, lane, t);
        }
      }
      flush_sec(fb);
      if (lane == 0) A.counters[(int64_t)tile * P.n_groups + it.group] = 0u;
    }
  }
}


// Distribute kernel instantiations (MODE): kPlain for plans with stored
// clique tables and no fused items, at the plain item's register budget
// and occupancy; kFused for plans whose work lists hold fused items;
// kRecomp for plans that recompute their clique tables (the collect
// kernel's register budget and per-warp map memory).
enum { kPlain = 0, kFused = 1, kRecomp = 2 };
constexpr int dist_blocks_per_sm(int mode) {
  return mode == kFused ? kFusedBlocksPerSM : mode == kRecomp ? kCollectBlocksPerSM : kDistributeBlocksPerSM;
}

// The warp's dynamic shared memory: fused secondary sums, or the clique's
// maps when recomputing.
template <int CPT, int MODE>
__device__ __forceinline__ unsigned char *dist_warp_smem(const DevPlan &P, unsigned char *dsm, int warp) {
  if constexpr (MODE == kFused) return dsm + (size_t)warp * P.sec_rows * (32 * CPT) * sizeof(float);
  else if constexpr (MODE == kRecomp) return dsm + (size_t)warp * collect_warp_smem(CPT, P.max_maps);
  else return dsm;
}

template <int CPT, int MODE, LoadMode RHO>
__device__ __forceinline__ void dist_unit(const DevPlan &P, const DevArena &A, const DItem &it, int tile, int lane,
                                          unsigned char *ws) {
  if constexpr (MODE == kFused) distribute_pair_item<CPT, RHO>(P, A, it, tile, lane, reinterpret_cast<float *>(ws));
  else if constexpr (MODE == kRecomp) distribute_item<CPT, RHO, true>(P, A, it, tile, lane, ws);
  else distribute_item<CPT, RHO>(P, A, it, tile, lane);
}

template <int CPT, int MODE>
__global__ void __launch_bounds__(kThreads, dist_blocks_per_sm(MODE))
    k_distribute(DevPlan P, DevArena A, int64_t item_begin, int64_t n_items) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t iw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (iw >= n_items) return;
  dist_unit<CPT, MODE, LD_NC>(P, A, P.ditems[item_begin + iw], blockIdx.y, lane, dist_warp_smem<CPT, MODE>(P, dsm, warp));
}

// ---------------------------------------------------------------------------
// dataflow schedule: one persistent launch per pass
// ---------------------------------------------------------------------------
//
// Case tiles are independent, so a clique's collect work on tile k needs
// only its children's collect work on tile k, and a clique's distribute
// work on tile k only its parent's task for it on tile k.  A pass is one
// launch: warps take units (work item, tile) from a global counter in tree
// order (collect: deepest layer first; distribute: root first; tile-major
// inside a layer), wait until the unit's producers on its tile have
// finished (per-(tile, clique) counters), do the item, and count it done.
// A unit only waits for units taken before it, and every taken unit is held
// by a running warp, so the pass always completes.  Waits are bounded: a
// wait that runs out sets the arena's error flag, every other wait then
// gives up at once, and the host reports JT_ETIMEOUT (limit: the plan's
// wait_limit_us, 2 s by default).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Lane 0 waits until *ctr >= need and fences (acquire: the producers'
// writes made before their counter increments are visible to it); the warp
// barrier then orders those writes before every lane's later loads.
__device__ __forceinline__ bool wait_ready(const uint32_t *ctr, uint32_t need, uint32_t *errflag, uint64_t limit_ns,
                                           int lane) {
  int ok = 1;
  if (lane == 0) {
    const volatile uint32_t *vc = ctr;
    const volatile uint32_t *ve = errflag;
    if (*vc < need) {
      const unsigned long long t0 = global_ns();
      unsigned ns = 32;
      while (*vc < need) {
        if (*ve != 0u) { ok = 0; break; }
        if (global_ns() - t0 > limit_ns) {
          atomicOr(errflag, 1u);
          ok = 0;
          break;
        }
        __nanosleep(ns);
        if (ns < 1024) ns *= 2;
      }
    }
    __threadfence();
  }
  __syncwarp();
  ok = __shfl_sync(kFull, ok, 0);
  return ok != 0;
}

// A unit is done: every lane's writes are fenced, the warp synchronises, and
// lane 0 publishes with a release (fence, then the counter increment).
__device__ __forceinline__ void signal_done(uint32_t *ctr, int lane) {
  __threadfence();
  __syncwarp();
  if (lane == 0 && ctr != nullptr) {
    __threadfence();
    atomicAdd(ctr, 1u);
  }
}

// Next unit of a pass: returns false when the pass is exhausted; else the
// item index and tile.  pref[k] = items of flow layers before k, begin[k]
// = the first item of flow layer k in the pass's item list.
__device__ __forceinline__ bool next_unit(unsigned long long *queue, const int64_t *pref, const int64_t *begin,
                                          int n_layers, int tiles, int lane, int64_t &item, int &tile) {
  long long u = 0;
  if (lane == 0) u = (long long)atomicAdd(queue, 1ull);
  u = __shfl_sync(kFull, u, 0);
  if (u >= pref[n_layers] * (long long)tiles) return false;
  const long long q = u / tiles;
  int lo = 0, hi = n_layers - 1;  // largest k with pref[k] <= q
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pref[mid] <= q) lo = mid; else hi = mid - 1;
  }
  const long long local = u - pref[lo] * (long long)tiles;
  const long long nk = pref[lo + 1] - pref[lo];
  tile = (int)(local / nk);
  item = begin[lo] + (local - (long long)tile * nk);
  return true;
}

template <int CPT, bool SLICED>
__global__ void __launch_bounds__(kThreads, kCollectBlocksPerSM) k_collect_flow(DevPlan P, DevArena A, int max_maps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char *ws = smem_raw + (size_t)warp * collect_warp_smem(CPT, max_maps);
  int64_t item;
  int tile;
  while (next_unit(A.queue, P.c_flow_pref, P.c_flow_begin, P.n_flow_layers, A.tiles, lane, item, tile)) {
    const DItem it = P.citems[item];
    uint32_t *ready = A.ready + (int64_t)tile * 2 * P.n_cliques;
    const uint32_t need = P.c_need[it.task];
    if (need == 0u || wait_ready(ready + it.task, need, A.errflag, P.wait_limit_ns, lane))
      collect_item<CPT, LD_PLAIN, SLICED>(P, A, it, tile, ws, max_maps, lane);
    const int parent = P.c_notify[it.task];
    signal_done(parent >= 0 ? ready + parent : nullptr, lane);
  }
}

template <int CPT, int MODE>
__global__ void __launch_bounds__(kThreads, dist_blocks_per_sm(MODE)) k_distribute_flow(DevPlan P, DevArena A) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int lane = threadIdx.x & 31;
  int64_t item;
  int tile;
  while (next_unit(A.queue + 16, P.d_flow_pref, P.d_flow_begin, P.n_flow_layers, A.tiles, lane, item, tile)) {
    {
      // nothing of the scheduling is kept in registers through the item
      const DItem &it = P.ditems[item];
      const uint32_t c = P.tasks[it.task].clique;
      const uint32_t need = P.d_need[c];
      if (need == 0u ||
          wait_ready(A.ready + ((int64_t)tile * 2 + 1) * P.n_cliques + c, need, A.errflag, P.wait_limit_ns, lane))
        dist_unit<CPT, MODE, LD_PLAIN>(P, A, it, tile, lane, dist_warp_smem<CPT, MODE>(P, dsm, threadIdx.x >> 5));
    }
    const DItem &it = P.ditems[item];
    const DTask &T = P.tasks[it.task];
    uint32_t *ready = A.ready + ((int64_t)tile * 2 + 1) * P.n_cliques;
    // a fused item also completes its share of the secondary child's ratio
    if (MODE == kFused && it.fused && T.sec_kind == TASK_CHILD) {
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicAdd(ready + T.sec_dst, 1u);
    }
    signal_done(T.kind == TASK_CHILD ? ready + T.dst : nullptr, lane);
  }
}

// ---------------------------------------------------------------------------
// explicit unit lists (iteration-level batching of the serving loop): one
// launch per pass covers a list of (work item, tile) units, each tile of the
// list at its own tree layer; a warp takes one unit.
// ---------------------------------------------------------------------------
template <int CPT, bool SLICED>
__global__ void __launch_bounds__(kThreads, kCollectBlocksPerSM) k_collect_units(DevPlan P, DevArena A, const int2 *units,
                                                                                 int n_units, int max_maps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (u >= n_units) return;
  const int2 un = units[u];
  collect_item<CPT, LD_NC, SLICED>(P, A, P.citems[un.x], un.y,
                                   smem_raw + (size_t)warp * collect_warp_smem(CPT, max_maps), max_maps, lane);
}

template <int CPT, int MODE>
__global__ void __launch_bounds__(kThreads, dist_blocks_per_sm(MODE))
    k_distribute_units(DevPlan P, DevArena A, const int2 *units, int n_units) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  if (u >= n_units) return;
  const int2 un = units[u];
  dist_unit<CPT, MODE, LD_NC>(P, A, P.ditems[un.x], un.y, lane, dist_warp_smem<CPT, MODE>(P, dsm, warp));
}

// ---------------------------------------------------------------------------
// finalize, part 1: log P(e) and status, one thread per case
// ---------------------------------------------------------------------------
constexpr int kStageCols = 16;

// k_logpe: a block holds 32 cases x kLogpeSlices slices.  Phase 1 finds,
// per case, the components holding an observed variable (a bitmask per
// component in shared memory); phase 2 spreads every observed component's
// terms -- the root total's log and base exponent, the other cliques'
// message exponents -- over the slices; a fixed-order sum over the slices
// gives each case's log P(e).
constexpr int kLogpeSlices = 32;

__global__ void k_logpe(DevPlan P, DevArena A, int W, int32_t n_cases, double *__restrict__ log_pe,
                        int32_t *__restrict__ status) {
  extern __shared__ unsigned char logpe_smem[];
  double *s_lz = reinterpret_cast<double *>(logpe_smem);              // [slice][32]
  long long *s_K = reinterpret_cast<long long *>(s_lz + kLogpeSlices * 32);
  int *s_zero = reinterpret_cast<int *>(s_K + kLogpeSlices * 32);
  unsigned *s_obs = reinterpret_cast<unsigned *>(s_zero + kLogpeSlices * 32);  // [n_comp], bit c = case c
  const int c = threadIdx.x;      // case within the block
  const int slice = threadIdx.y;
  const int64_t cs = (int64_t)blockIdx.x * 32 + c;
  const int tile = (int)(cs / W), col = (int)(cs - (int64_t)tile * W);
  for (int q = slice * 32 + c; q < P.n_comp; q += 32 * kLogpeSlices) s_obs[q] = 0u;
  __syncthreads();
  // phase 1: components with an observed variable (a component without one
  // has probability exactly 1: a sum over all states of a product of CPTs);
  // the (component, variable) pairs are spread over the slices
  for (int k = slice; k < P.n_comp_vars; k += kLogpeSlices)
    if (A.ev[((int64_t)tile * P.n_vars + P.comp_vars[k]) * W + col] >= 0) {
      const int q = P.comp_var_owner[k];
      if (!((s_obs[q] >> c) & 1u)) atomicOr(&s_obs[q], 1u << c);
    }
  __syncthreads();
  // phase 2: messages multiplied into a parent were scaled by 2^-k, so k is
  // added back; every observed component root adds the log of its total
  long long K = 0;
  double lz = 0.0;
  int zero = 0;
  for (int q = slice; q < P.n_comp; q += kLogpeSlices) {
    if (!((s_obs[q] >> c) & 1u)) continue;
    const DClique &D = P.cl[P.comp_roots[q]];
    const float z = A.phistar[((int64_t)tile * P.sep_rows + D.sep_row) * W + col];
    if (z > 0.f) lz += log((double)z); else zero = 1;
    K += D.comp_base_exp;
  }
  for (int k = slice; P.rescale && k < P.n_comp_cliques; k += kLogpeSlices) {
    if (!((s_obs[P.comp_owner[k]] >> c) & 1u)) continue;
    K += pow2_exp(A.maxbits[((int64_t)tile * P.n_cliques + P.comp_cliques[k]) * W + col]);
  }
  s_lz[slice * 32 + c] = lz;
  s_K[slice * 32 + c] = K;
  s_zero[slice * 32 + c] = zero;
  __syncthreads();
  if (slice != 0 || cs >= n_cases) return;
  for (int t = 1; t < kLogpeSlices; ++t) {
    lz += s_lz[t * 32 + c];
    K += s_K[t * 32 + c];
    zero |= s_zero[t * 32 + c];
  }
  const int bad = A.bad[cs];
  const bool incomplete = *reinterpret_cast<volatile const uint32_t *>(A.errflag) != 0u;
  const int st = incomplete ? JT_CASE_INCOMPLETE
                            : bad ? JT_CASE_BAD_EVIDENCE : (zero ? JT_CASE_ZERO_EVIDENCE : JT_CASE_OK);
  double lp;
  if (st == JT_CASE_OK) lp = lz + (double)K * 0.69314718055994530942;
  else if (st == JT_CASE_ZERO_EVIDENCE) lp = -INFINITY;
  else lp = NAN;
  log_pe[cs] = lp;
  status[cs] = st;
}

__global__ void k_posterior(DevPlan P, DevArena A, int W, int32_t n_cases, const int32_t *__restrict__ status,
                            double *__restrict__ post) {
  extern __shared__ double stage[];  // [W][kStageCols + 1], then float [kStageCols][W] inputs
  const int tile = blockIdx.x;
  const int c = threadIdx.x;
  const int64_t cs = (int64_t)tile * W + c;
  const int64_t left = (int64_t)n_cases - (int64_t)tile * W;
  const int rows_here = (int)(left < W ? left : W);
  if ((int)blockIdx.y >= P.n_pgroups) {  // pruned plan: columns of the removed variables
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int rr = warp; rr < rows_here; rr += nw)
      for (int k = lane; k < P.n_nan_cols; k += 32)
        post[((int64_t)tile * W + rr) * P.io_post_rows + P.io_nan_cols[k]] = NAN;
    return;
  }
  const int st = cs < n_cases ? status[cs] : JT_CASE_BAD_EVIDENCE;
  const int v0 = P.pgroup_ptr[blockIdx.y], v1 = P.pgroup_ptr[blockIdx.y + 1];
  int64_t col0 = P.post_off[v0];  // first column of the staged block
  auto flush = [&](int ncols) {
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int rr = warp; rr < rows_here; rr += nw)
      for (int j = lane; j < ncols; j += 32)
        post[((int64_t)tile * W + rr) * P.io_post_rows + (P.io_post_col ? P.io_post_col[col0 + j] : col0 + j)] =
            stage[rr * (kStageCols + 1) + j];
    __syncthreads();
  };
  const int ncols_all = (int)(P.post_off[v1 - 1] + P.card[v1 - 1] - col0);
  if (ncols_all <= kStageCols) {
    // every input of the group requested at once (one load each, no chain
    // of dependent loads), then normalised from shared memory; each thread
    // touches only its own case's column of `in`
    float *in = reinterpret_cast<float *>(stage + (size_t)W * (kStageCols + 1));
    const float *m0 = A.post + ((int64_t)tile * P.post_rows + col0) * W + c;
    float x[kStageCols];
    int e[kStageCols];
#pragma unroll
    for (int j = 0; j < kStageCols; ++j) x[j] = j < ncols_all ? m0[(int64_t)j * W] : 0.f;
#pragma unroll
    for (int k = 0; k < kStageCols; ++k) e[k] = v0 + k < v1 ? A.ev[((int64_t)tile * P.n_vars + v0 + k) * W + c] : -1;
#pragma unroll
    for (int j = 0; j < kStageCols; ++j) in[j * W + c] = x[j];
#pragma unroll
    for (int k = 0; k < kStageCols; ++k) {
      if (v0 + k < v1) {  // the same for every thread of the block
        const int o = (int)(P.post_off[v0 + k] - col0);
        const int r = P.card[v0 + k];
        double s = 0.0;
        if (st == JT_CASE_OK && e[k] < 0)
          for (int j = 0; j < r; ++j) s += (double)in[(o + j) * W + c];
        const double inv = 1.0 / s;
        for (int j = 0; j < r; ++j) {
          double val;
          if (st != JT_CASE_OK) val = NAN;
          else if (e[k] >= 0) val = (j == e[k]) ? 1.0 : 0.0;
          else val = (double)in[(o + j) * W + c] * inv;
          stage[c * (kStageCols + 1) + o + j] = val;
        }
      }
    }
    flush(ncols_all);
    return;
  }
  for (int v = v0; v < v1; ++v) {  // a variable with more than kStageCols states
    const int64_t off = P.post_off[v];
    const int r = P.card[v];
    const int ev = A.ev[((int64_t)tile * P.n_vars + v) * W + c];
    const float *m = A.post + ((int64_t)tile * P.post_rows + off) * W + c;
    // FP64 sum and one FP64 reciprocal per variable (FP64 division is slow
    // on this part; m * (1/s) differs from m / s by at most an FP64 ulp)
    double s = 0.0;
    if (st == JT_CASE_OK && ev < 0)
      for (int j = 0; j < r; ++j) s += (double)m[(int64_t)j * W];
    const double inv = 1.0 / s;
    for (int j = 0; j < r; ++j) {
      if (off + j - col0 == kStageCols) {
        flush(kStageCols);
        col0 += kStageCols;
      }
      double val;
      if (st != JT_CASE_OK) val = NAN;
      else if (ev >= 0) val = (j == ev) ? 1.0 : 0.0;
      else val = (double)m[(int64_t)j * W] * inv;
      stage[c * (kStageCols + 1) + (off + j - col0)] = val;
    }
  }
  flush((int)(P.post_off[v1 - 1] + P.card[v1 - 1] - col0));
}

// ---------------------------------------------------------------------------
// plain FP64 path: one thread per table entry, div/mod indices, atomics
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t plain_index(int64_t e, const int64_t *q, int nv) {
  int64_t idx = 0;
  for (int i = 0; i < nv; ++i) idx += ((e / q[4 * i + 2]) % q[4 * i + 1]) * q[4 * i + 3];
  return idx;
}

__global__ void k_plain_init(double *psi, const double *base, DPlainMap m, const int64_t *pool,
                             const int32_t *ev) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.size) return;
  const int64_t *q = pool + m.var_off;
  double val = base[e];
  for (int i = 0; i < m.nv; ++i) {
    const int v = (int)q[4 * i];
    const int d = (int)((e / q[4 * i + 2]) % q[4 * i + 1]);
    const int x = ev[v];
    if (x >= 0 && x != d) val = 0.0;
  }
  psi[e] = val;
}

__global__ void k_plain_marg(const double *src, double *dst, DPlainMap m, const int64_t *pool) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.size) return;
  atomicAdd(dst + plain_index(e, pool + m.var_off, m.nv), src[e]);
}

__global__ void k_plain_extend(double *x, const double *y, DPlainMap m, const int64_t *pool) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.size) return;
  x[e] *= y[plain_index(e, pool + m.var_off, m.nv)];
}

__global__ void k_plain_divide(double *num, const double *den, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  num[i] = (den[i] != 0.0) ? num[i] / den[i] : 0.0;
}

__global__ void k_plain_finalize(const double *pe, const double *marg, const int32_t *ev,
                                 const int32_t *card, const int64_t *post_off, int32_t n_vars,
                                 double *log_pe, double *post, int32_t *status) {
  const double z = *pe;
  const int st = z > 0.0 ? JT_CASE_OK : JT_CASE_ZERO_EVIDENCE;
  if (threadIdx.x == 0) {
    *log_pe = st == JT_CASE_OK ? log(z) : -INFINITY;
    *status = st;
  }
  for (int v = threadIdx.x; v < n_vars; v += blockDim.x) {
    const int64_t off = post_off[v];
    const int r = card[v];
    if (st != JT_CASE_OK) {
      for (int j = 0; j < r; ++j) post[off + j] = NAN;
    } else if (ev[v] >= 0) {
      for (int j = 0; j < r; ++j) post[off + j] = (j == ev[v]) ? 1.0 : 0.0;
    } else {
      double s = 0.0;
      for (int j = 0; j < r; ++j) s += marg[off + j];
      for (int j = 0; j < r; ++j) post[off + j] = marg[off + j] / s;
    }
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

size_t collect_smem_bytes(int cpt, int max_maps) {
  return std::min<size_t>(kWarps * collect_warp_smem(cpt, max_maps), kCollectSmemLimit);
}
size_t collect_warp_smem_bytes(int cpt, int max_maps) { return collect_warp_smem(cpt, max_maps); }

void launch_evidence(int cpt, const int32_t *d_ev_in, int32_t n_cases, const DevPlan &P,
                     const DevArena &A, cudaStream_t s) {
  const int W = 32 * cpt;
  const dim3 grid((unsigned)(((int64_t)A.tiles * W + 31) / 32),
                  (unsigned)((P.n_vars + 31) / 32 + (P.n_dropped + 31) / 32));
  k_evidence<<<grid, dim3(32, 8), 0, s>>>(d_ev_in, n_cases, P, A, W);
}

// Warps per collect block: eight, fewer when a layer's cliques carry so many
// maps that eight warps' shared memory would not fit.
static int collect_warps(int cpt, int max_maps) {
  const size_t per_warp = collect_warp_smem(cpt, max_maps);
  return (int)std::min<size_t>(kWarps, std::max<size_t>(1, kCollectSmemLimit / std::max<size_t>(per_warp, 1)));
}

size_t distribute_smem_bytes(int cpt, int sec_rows) {
  return (size_t)kWarps * (size_t)sec_rows * 32 * (size_t)cpt * sizeof(float);
}

// Calls f(CPT, MODE) with both as compile-time constants.
template <class F>
static auto with_distribute(int cpt, int mode, F &&f) {
  using std::integral_constant;
  auto by_mode = [&](auto c) {
    if (mode == kFused) return f(c, integral_constant<int, kFused>{});
    if (mode == kRecomp) return f(c, integral_constant<int, kRecomp>{});
    return f(c, integral_constant<int, kPlain>{});
  };
  if (cpt == 8) return by_mode(integral_constant<int, 8>{});
  if (cpt == 4) return by_mode(integral_constant<int, 4>{});
  if (cpt == 2) return by_mode(integral_constant<int, 2>{});
  return by_mode(integral_constant<int, 1>{});
}

static int dist_mode(const DevPlan &P) {
  return P.recompute ? kRecomp : P.fused_items > 0 ? kFused : kPlain;
}

// Dynamic shared memory of a distribute block in a mode.
static size_t dist_smem(int cpt, int mode, int sec_rows, int max_maps) {
  if (mode == kFused) return distribute_smem_bytes(cpt, sec_rows);
  if (mode == kRecomp) return (size_t)kWarps * collect_warp_smem(cpt, max_maps);
  return 0;
}

// Calls f(CPT, SLICED) with both as compile-time constants: the collect
// kernels are instantiated per cases-per-thread and per plan kind.
template <class F>
static auto with_collect(int cpt, bool sliced, F &&f) {
  using std::integral_constant;
  using yes = std::true_type;
  using no = std::false_type;
  if (cpt == 8) return sliced ? f(integral_constant<int, 8>{}, yes{}) : f(integral_constant<int, 8>{}, no{});
  if (cpt == 4) return sliced ? f(integral_constant<int, 4>{}, yes{}) : f(integral_constant<int, 4>{}, no{});
  if (cpt == 2) return sliced ? f(integral_constant<int, 2>{}, yes{}) : f(integral_constant<int, 2>{}, no{});
  return sliced ? f(integral_constant<int, 1>{}, yes{}) : f(integral_constant<int, 1>{}, no{});
}

static bool is_sliced(const DevPlan &P) { return P.slice_var != nullptr; }

cudaError_t configure_collect_smem(int cpt, bool sliced, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return with_collect(cpt, sliced, [&](auto c, auto sl) {
    constexpr int CPT = decltype(c)::value;
    constexpr bool SL = decltype(sl)::value;
    cudaError_t e =
        cudaFuncSetAttribute((const void *)k_collect<CPT, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void *)k_collect_units<CPT, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k_collect_flow<CPT, SL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
  });
}

void launch_collect_units(int cpt, const DevPlan &P, const DevArena &A, const int2 *units, int n_units, int max_maps,
                          cudaStream_t s) {
  if (n_units <= 0) return;
  with_collect(cpt, is_sliced(P), [&](auto c, auto sl) {
    constexpr int CPT = decltype(c)::value;
    const int nw = collect_warps(CPT, max_maps);
    const size_t smem = (size_t)nw * collect_warp_smem(CPT, max_maps);
    k_collect_units<CPT, decltype(sl)::value><<<(unsigned)((n_units + nw - 1) / nw), 32 * nw, smem, s>>>(
        P, A, units, n_units, max_maps);
  });
}

void launch_distribute_units(int cpt, const DevPlan &P, const DevArena &A, const int2 *units, int n_units,
                             cudaStream_t s) {
  if (n_units <= 0) return;
  const unsigned grid = (unsigned)((n_units + kWarps - 1) / kWarps);
  const int mode = dist_mode(P);
  const size_t sm = dist_smem(cpt, mode, P.sec_rows, P.max_maps);
  with_distribute(cpt, mode, [&](auto c, auto m) {
    k_distribute_units<decltype(c)::value, decltype(m)::value><<<grid, kThreads, sm, s>>>(P, A, units, n_units);
  });
}

void launch_collect(int cpt, const DevPlan &P, const DevArena &A, int64_t b, int64_t n, int max_maps,
                    cudaStream_t s) {
  if (n <= 0) return;
  with_collect(cpt, is_sliced(P), [&](auto c, auto sl) {
    constexpr int CPT = decltype(c)::value;
    const int nw = collect_warps(CPT, max_maps);
    const size_t smem = (size_t)nw * collect_warp_smem(CPT, max_maps);
    dim3 grid((unsigned)((n + nw - 1) / nw), (unsigned)A.tiles);
    k_collect<CPT, decltype(sl)::value><<<grid, 32 * nw, smem, s>>>(P, A, b, n, max_maps);
  });
}



cudaError_t configure_distribute_smem(int cpt, int sec_rows, int max_maps) {
  for (int mode : {kFused, kRecomp}) {
    const size_t bytes = dist_smem(cpt, mode, sec_rows, max_maps);
    if (bytes <= 48 * 1024) continue;
    const cudaError_t e = with_distribute(cpt, mode, [&](auto c, auto m) {
      constexpr int CPT = decltype(c)::value;
      constexpr int MODE = decltype(m)::value;
      cudaError_t r = cudaFuncSetAttribute((const void *)k_distribute<CPT, MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (r != cudaSuccess) return r;
      r = cudaFuncSetAttribute((const void *)k_distribute_units<CPT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bytes);
      if (r != cudaSuccess) return r;
      return cudaFuncSetAttribute((const void *)k_distribute_flow<CPT, MODE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void launch_distribute(int cpt, const DevPlan &P, const DevArena &A, int64_t b, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  dim3 grid((unsigned)((n + kWarps - 1) / kWarps), (unsigned)A.tiles);
  const int mode = dist_mode(P);
  const size_t sm = dist_smem(cpt, mode, P.sec_rows, P.max_maps);
  with_distribute(cpt, mode, [&](auto c, auto m) {
    k_distribute<decltype(c)::value, decltype(m)::value><<<grid, kThreads, sm, s>>>(P, A, b, n);
  });
}

void launch_collect_flow(int cpt, const DevPlan &P, const DevArena &A, int blocks, int max_maps, cudaStream_t s) {
  with_collect(cpt, is_sliced(P), [&](auto c, auto sl) {
    constexpr int CPT = decltype(c)::value;
    const int nw = collect_warps(CPT, max_maps);
    const size_t smem = (size_t)nw * collect_warp_smem(CPT, max_maps);
    k_collect_flow<CPT, decltype(sl)::value><<<blocks, 32 * nw, smem, s>>>(P, A, max_maps);
  });
}

void launch_distribute_flow(int cpt, const DevPlan &P, const DevArena &A, int blocks, cudaStream_t s) {
  const int mode = dist_mode(P);
  const size_t sm = dist_smem(cpt, mode, P.sec_rows, P.max_maps);
  with_distribute(cpt, mode, [&](auto c, auto m) {
    k_distribute_flow<decltype(c)::value, decltype(m)::value><<<blocks, kThreads, sm, s>>>(P, A);
  });
}

// Resident blocks per SM of the dataflow kernels (their grids fill the GPU once).
template <class K>
static int occupancy_of(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

int flow_blocks_per_sm(int cpt, bool sliced, int max_maps) {
  const int nw = collect_warps(cpt, max_maps);
  const size_t smem = (size_t)nw * collect_warp_smem(cpt, max_maps);
  return with_collect(cpt, sliced, [&](auto c, auto sl) {
    return occupancy_of(k_collect_flow<decltype(c)::value, decltype(sl)::value>, 32 * nw, smem);
  });
}

int distribute_flow_blocks_per_sm(int cpt, const DevPlan &P) {
  const int mode = dist_mode(P);
  const size_t sm = dist_smem(cpt, mode, P.sec_rows, P.max_maps);
  return with_distribute(cpt, mode, [&](auto c, auto m) {
    return occupancy_of(k_distribute_flow<decltype(c)::value, decltype(m)::value>, kThreads, sm);
  });
}

size_t recompute_warp_smem_bytes(int cpt, int max_maps) { return collect_warp_smem(cpt, max_maps); }

void launch_plain_init(double *psi, const double *base, const DPlainMap &m, const int64_t *pool,
                       const int32_t *d_ev, cudaStream_t s) {
  k_plain_init<<<blocks_for(m.size, 256), 256, 0, s>>>(psi, base, m, pool, d_ev);
}
void launch_plain_marg(const double *src, double *dst, const DPlainMap &m, const int64_t *pool,
                       cudaStream_t s) {
  k_plain_marg<<<blocks_for(m.size, 256), 256, 0, s>>>(src, dst, m, pool);
}
void launch_plain_extend(double *x, const double *y, const DPlainMap &m, const int64_t *pool,
                         cudaStream_t s) {
  k_plain_extend<<<blocks_for(m.size, 256), 256, 0, s>>>(x, y, m, pool);
}
void launch_plain_divide(double *num, const double *den, int64_t n, cudaStream_t s) {
  k_plain_divide<<<blocks_for(n, 256), 256, 0, s>>>(num, den, n);
}
void launch_plain_finalize(const double *pe, const double *marg, const int32_t *d_ev,
                           const int32_t *card, const int64_t *post_off, int32_t n_vars,
                           double *d_log_pe, double *d_post, int32_t *d_status, cudaStream_t s) {
  k_plain_finalize<<<1, 256, 0, s>>>(pe, marg, d_ev, card, post_off, n_vars, d_log_pe, d_post, d_status);
}

size_t logpe_smem_bytes(int n_comp) {
  return (sizeof(double) + sizeof(long long) + sizeof(int)) * kLogpeSlices * 32 +
         sizeof(unsigned) * (size_t)std::max(1, n_comp);
}

cudaError_t configure_logpe_smem(int n_comp) {
  const size_t bytes = logpe_smem_bytes(n_comp);
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(k_logpe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t posterior_smem_bytes(int W) {
  return sizeof(double) * (size_t)W * (kStageCols + 1) + sizeof(float) * (size_t)kStageCols * W;
}

cudaError_t configure_posterior_smem() {
  return cudaFuncSetAttribute(k_posterior, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)posterior_smem_bytes(32 * 8));
}

void launch_finalize(int cpt, const DevPlan &P, const DevArena &A, int32_t n_cases,
                     int64_t root_sep_row, double *d_log_pe, double *d_post, int32_t *d_status,
                     cudaStream_t s) {
  (void)root_sep_row;
  if (n_cases <= 0) return;
  const int W = 32 * cpt;
  const unsigned tiles = (unsigned)((n_cases + W - 1) / W);
  const size_t lsmem = logpe_smem_bytes(P.n_comp);
  k_logpe<<<(unsigned)((n_cases + 31) / 32), dim3(32, kLogpeSlices), lsmem, s>>>(P, A, W, n_cases, d_log_pe, d_status);
  const size_t smem = posterior_smem_bytes(W);
  k_posterior<<<dim3(tiles, (unsigned)(P.n_pgroups + (P.n_nan_cols > 0))), W, smem, s>>>(P, A, W, n_cases,
                                                                                         d_status, d_post);
}

}  // namespace jt
