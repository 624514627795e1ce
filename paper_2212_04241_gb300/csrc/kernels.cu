// Message kernels of the batched FP32 junction-tree path and of the plain
// FP64 comparator path.
//
// Batched path.  One launch per tree layer and pass covers every clique of
// that layer (Section 2: BFS layers, all table entries of a layer packed
// into one parallel task) for every evidence case of the chunk: the grid is
// (thread blocks of the layer's work list) x (case tiles).  Tables are
// [tile][row][W] with W = 32 * CPT consecutive cases per row, so every index
// computation is uniform across a warp and amortised over W cases, and every
// row access is a fully coalesced W*4-byte transaction.
//
//   collect (Section 2: reduction + extension + marginalisation, fused):
//     psi_C[e] = base_C[e] * [evidence of homed variables] *
//                prod_children phi*_child[map(e)] * 2^-k_child
//     phi*_C[s] = sum_u psi_C[s*R + u]          (upward separator outermost)
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

#include "kernels.cuh"

namespace jt {
namespace {

template <int CPT>
struct Vec {
  float x[CPT];
};

template <int CPT>
__device__ __forceinline__ Vec<CPT> vzero() {
  Vec<CPT> r;
#pragma unroll
  for (int k = 0; k < CPT; ++k) r.x[k] = 0.f;
  return r;
}

template <int CPT>
__device__ __forceinline__ Vec<CPT> ld_plain(const float *p) {
  Vec<CPT> r;
  if constexpr (CPT == 4) {
    float4 t = *reinterpret_cast<const float4 *>(p);
    r.x[0] = t.x; r.x[1] = t.y; r.x[2] = t.z; r.x[3] = t.w;
  } else if constexpr (CPT == 2) {
    float2 t = *reinterpret_cast<const float2 *>(p);
    r.x[0] = t.x; r.x[1] = t.y;
  } else {
    r.x[0] = *p;
  }
  return r;
}

// read-once data (streamed from HBM)
template <int CPT>
__device__ __forceinline__ Vec<CPT> ld_stream(const float *p) {
  Vec<CPT> r;
  if constexpr (CPT == 4) {
    float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    r.x[0] = t.x; r.x[1] = t.y; r.x[2] = t.z; r.x[3] = t.w;
  } else if constexpr (CPT == 2) {
    float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
    r.x[0] = t.x; r.x[1] = t.y;
  } else {
    r.x[0] = __ldcs(p);
  }
  return r;
}

// data written by other blocks of the same launch: bypass L1
template <int CPT>
__device__ __forceinline__ Vec<CPT> ld_cg(const float *p) {
  Vec<CPT> r;
  if constexpr (CPT == 4) {
    float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
    r.x[0] = t.x; r.x[1] = t.y; r.x[2] = t.z; r.x[3] = t.w;
  } else if constexpr (CPT == 2) {
    float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
    r.x[0] = t.x; r.x[1] = t.y;
  } else {
    r.x[0] = __ldcg(p);
  }
  return r;
}

template <int CPT>
__device__ __forceinline__ void st_plain(float *p, const Vec<CPT> &v) {
  if constexpr (CPT == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(v.x[0], v.x[1], v.x[2], v.x[3]);
  } else if constexpr (CPT == 2) {
    *reinterpret_cast<float2 *>(p) = make_float2(v.x[0], v.x[1]);
  } else {
    *p = v.x[0];
  }
}

// write-once data that is read back only much later
template <int CPT>
__device__ __forceinline__ void st_stream(float *p, const Vec<CPT> &v) {
  if constexpr (CPT == 4) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v.x[0], v.x[1], v.x[2], v.x[3]));
  } else if constexpr (CPT == 2) {
    __stcs(reinterpret_cast<float2 *>(p), make_float2(v.x[0], v.x[1]));
  } else {
    __stcs(p, v.x[0]);
  }
}

// Compensated (Kahan) accumulation per case: long FP32 sums keep ~2 ulp.
template <int CPT>
__device__ __forceinline__ void kahan_add(Vec<CPT> &sum, Vec<CPT> &comp, const Vec<CPT> &v) {
#pragma unroll
  for (int k = 0; k < CPT; ++k) {
    float y = v.x[k] - comp.x[k];
    float t = sum.x[k] + y;
    comp.x[k] = (t - sum.x[k]) - y;
    sum.x[k] = t;
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
__global__ void k_evidence(const int32_t *__restrict__ ev_in, int32_t n_cases, DevPlan P,
                           DevArena A, int W) {
  const int64_t total = (int64_t)A.tiles * W * P.n_vars;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / P.n_vars;
    const int v = (int)(i - c * P.n_vars);
    int val = -1;
    if (c < n_cases) {
      val = ev_in[c * P.n_vars + v];
      if (val < -1 || val >= P.card[v]) {
        A.bad[c] = 1;
        val = -1;
      }
    }
    A.ev[((c / W) * P.n_vars + v) * W + (c % W)] = val;
  }
}

// ---------------------------------------------------------------------------
// collect
// ---------------------------------------------------------------------------
struct CollectSmem {
  int64_t *mA, *mB, *mrow;
  float *mval, *red, *redm;
  int32_t *segA;
};

__host__ __device__ inline size_t collect_smem_layout(int cpt, int nm, CollectSmem *s, unsigned char *base) {
  const int W = 32 * cpt;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 15) & ~size_t(15);
    return o;
  };
  size_t oA = take(sizeof(int64_t) * nm), oB = take(sizeof(int64_t) * nm), oR = take(sizeof(int64_t) * nm);
  size_t oV = take(sizeof(float) * nm * W), oS = take(sizeof(float) * kWarps * W),
         oM = take(sizeof(float) * kWarps * W), oG = take(sizeof(int32_t) * kWarps * nm);
  if (s) {
    s->mA = reinterpret_cast<int64_t *>(base + oA);
    s->mB = reinterpret_cast<int64_t *>(base + oB);
    s->mrow = reinterpret_cast<int64_t *>(base + oR);
    s->mval = reinterpret_cast<float *>(base + oV);
    s->red = reinterpret_cast<float *>(base + oS);
    s->redm = reinterpret_cast<float *>(base + oM);
    s->segA = reinterpret_cast<int32_t *>(base + oG);
  }
  return off;
}

template <int CPT>
__global__ void __launch_bounds__(kThreads) k_collect(DevPlan P, DevArena A, int64_t item_begin) {
  constexpr int W = 32 * CPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_nchild;
  __shared__ int s_last;
  const DItem it = P.citems[item_begin + blockIdx.x];
  const int tile = blockIdx.y;
  const DClique C = P.cl[it.task];
  const int nm = C.map_end - C.map_begin;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  CollectSmem S;
  collect_smem_layout(CPT, nm, &S, smem_raw);

  for (int i = threadIdx.x; i < nm; i += kThreads) {
    const DMap mp = P.maps[C.map_begin + i];
    S.mA[i] = mp.A_off;
    S.mB[i] = mp.B_off;
    S.mrow[i] = ((int64_t)tile * P.sep_rows + mp.src_row) * W;
  }
  if (threadIdx.x == 0) {
    int k = 0;
    while (k < nm && P.maps[C.map_begin + k].kind == MAP_CHILD) ++k;
    s_nchild = k;
  }
  for (int i = threadIdx.x; i < nm * W; i += kThreads) {
    const int mi = i / W, c = i - mi * W;
    const DMap mp = P.maps[C.map_begin + mi];
    if (mp.kind == MAP_CHILD)
      S.mval[i] = pow2f(-pow2_exp(A.maxbits[((int64_t)tile * P.n_cliques + mp.src) * W + c]));
    else
      S.mval[i] = __int_as_float(A.ev[((int64_t)tile * P.n_vars + mp.src) * W + c]);
  }
  __syncthreads();
  const int nchild = s_nchild;
  const float *__restrict__ base = P.base32 + C.base_off;
  float *psi = A.psi + ((int64_t)tile * P.psi_rows + C.psi_row) * W + lane * CPT;
  const float *phs = A.phistar + lane * CPT;
  int32_t *segA = S.segA + warp * nm;

  Vec<CPT> mx = vzero<CPT>();
  auto load_segA = [&](int64_t s) {
    for (int i = lane; i < nm; i += 32) segA[i] = __ldg(P.ipool + S.mA[i] + s);
    __syncwarp();
  };
  auto rows = [&](int64_t s, int64_t ua, int64_t ub, Vec<CPT> &acc, Vec<CPT> &comp) {
    const int64_t e0 = s * C.R;
#pragma unroll 2
    for (int64_t u = ua; u < ub; ++u) {
      const int64_t e = e0 + u;
      const float b = __ldg(base + e);
      Vec<CPT> v;
#pragma unroll
      for (int k = 0; k < CPT; ++k) v.x[k] = b;
      for (int i = 0; i < nchild; ++i) {
        const int idx = segA[i] + __ldg(P.ipool + S.mB[i] + u);
        const Vec<CPT> m = ld_plain<CPT>(phs + S.mrow[i] + (int64_t)idx * W);
        const Vec<CPT> sc = ld_plain<CPT>(S.mval + i * W + lane * CPT);
#pragma unroll
        for (int k = 0; k < CPT; ++k) v.x[k] *= m.x[k] * sc.x[k];
      }
      for (int i = nchild; i < nm; ++i) {
        const int d = segA[i] + __ldg(P.ipool + S.mB[i] + u);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const int ev = __float_as_int(S.mval[i * W + lane * CPT + k]);
          if (ev >= 0 && ev != d) v.x[k] = 0.f;
        }
      }
      st_stream<CPT>(psi + e * W, v);
      kahan_add<CPT>(acc, comp, v);
    }
  };
  auto track_max = [&](const Vec<CPT> &m) {
#pragma unroll
    for (int k = 0; k < CPT; ++k) mx.x[k] = fmaxf(mx.x[k], m.x[k]);
  };

  float *phi_out = A.phistar + ((int64_t)tile * P.sep_rows + C.sep_row) * W + lane * CPT;
  if (!it.split) {
    for (int64_t s = it.t0 + warp; s < it.t0 + it.nt; s += kWarps) {
      load_segA(s);
      Vec<CPT> acc = vzero<CPT>(), comp = vzero<CPT>();
      rows(s, 0, C.R, acc, comp);
      st_plain<CPT>(phi_out + s * W, acc);
      track_max(acc);
      __syncwarp();
    }
  } else {
    const int64_t s = it.t0;
    const int64_t q = (it.nu + kWarps - 1) / kWarps;
    const int64_t ua = it.u0 + warp * q;
    const int64_t ub = min(ua + q, it.u0 + it.nu);
    load_segA(s);
    Vec<CPT> acc = vzero<CPT>(), comp = vzero<CPT>();
    if (ua < ub) rows(s, ua, ub, acc, comp);
    st_plain<CPT>(S.red + warp * W + lane * CPT, acc);
    __syncthreads();
    if (warp == 0) {
      Vec<CPT> tot = vzero<CPT>();
      for (int w = 0; w < kWarps; ++w) {
        const Vec<CPT> x = ld_plain<CPT>(S.red + w * W + lane * CPT);
#pragma unroll
        for (int k = 0; k < CPT; ++k) tot.x[k] += x.x[k];
      }
      if (it.npieces == 1) {
        st_plain<CPT>(phi_out + s * W, tot);
        track_max(tot);
      } else {
        st_plain<CPT>(A.partial + ((int64_t)tile * P.n_partials + it.partial) * W + lane * CPT, tot);
      }
    }
    if (it.npieces > 1) {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned old = atomicAdd(&A.counters[(int64_t)tile * P.n_groups + it.group], 1u);
        s_last = (old == (unsigned)(it.npieces - 1));
      }
      __syncthreads();
      if (s_last && warp == 0) {
        __threadfence();
        const int first = it.partial - it.piece;
        Vec<CPT> tot = vzero<CPT>();
        for (int p = 0; p < it.npieces; ++p) {
          const Vec<CPT> x = ld_cg<CPT>(A.partial + ((int64_t)tile * P.n_partials + first + p) * W + lane * CPT);
#pragma unroll
          for (int k = 0; k < CPT; ++k) tot.x[k] += x.x[k];
        }
        st_plain<CPT>(phi_out + s * W, tot);
        track_max(tot);
        if (lane == 0) A.counters[(int64_t)tile * P.n_groups + it.group] = 0u;
      }
    }
  }
  // per-case maximum of the message entries this block completed
  st_plain<CPT>(S.redm + warp * W + lane * CPT, mx);
  __syncthreads();
  if (warp == 0) {
    Vec<CPT> m = vzero<CPT>();
    for (int w = 0; w < kWarps; ++w) {
      const Vec<CPT> x = ld_plain<CPT>(S.redm + w * W + lane * CPT);
#pragma unroll
      for (int k = 0; k < CPT; ++k) m.x[k] = fmaxf(m.x[k], x.x[k]);
    }
    unsigned *mb = A.maxbits + ((int64_t)tile * P.n_cliques + it.task) * W + lane * CPT;
#pragma unroll
    for (int k = 0; k < CPT; ++k)
      if (m.x[k] > 0.f) atomicMax(mb + k, __float_as_uint(m.x[k]));
  }
}

// ---------------------------------------------------------------------------
// distribute
// ---------------------------------------------------------------------------
template <int CPT>
__global__ void __launch_bounds__(kThreads) k_distribute(DevPlan P, DevArena A, int64_t item_begin) {
  constexpr int W = 32 * CPT;
  __shared__ __align__(16) float red[kWarps * W];
  __shared__ int s_last;
  const DItem it = P.ditems[item_begin + blockIdx.x];
  const int tile = blockIdx.y;
  const DTask T = P.tasks[it.task];
  const DClique C = P.cl[T.clique];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float *psi = A.psi + ((int64_t)tile * P.psi_rows + C.psi_row) * W + lane * CPT;
  const float *rho = A.rho + ((int64_t)tile * P.sep_rows + C.sep_row) * W + lane * CPT;
  const bool root = C.is_root != 0;
  Vec<CPT> rs;
#pragma unroll
  for (int k = 0; k < CPT; ++k)
    rs.x[k] = root ? pow2f(-pow2_exp(A.maxbits[((int64_t)tile * P.n_cliques + T.clique) * W + lane * CPT + k]))
                   : 1.f;
  const int32_t *__restrict__ Bt = P.ipool + T.B_off;
  const int32_t *__restrict__ sBt = P.ipool + T.sB_off;

  auto rows = [&](int64_t t, int64_t ua, int64_t ub, Vec<CPT> &acc, Vec<CPT> &comp) {
    const int64_t a = __ldg(P.ipool + T.A_off + t);
    const int64_t sa = __ldg(P.ipool + T.sA_off + t);
    if (root) {
#pragma unroll 4
      for (int64_t u = ua; u < ub; ++u) {
        const Vec<CPT> p = ld_stream<CPT>(psi + (a + __ldg(Bt + u)) * W);
        Vec<CPT> v;
#pragma unroll
        for (int k = 0; k < CPT; ++k) v.x[k] = p.x[k] * rs.x[k];
        kahan_add<CPT>(acc, comp, v);
      }
    } else {
#pragma unroll 4
      for (int64_t u = ua; u < ub; ++u) {
        const Vec<CPT> p = ld_stream<CPT>(psi + (a + __ldg(Bt + u)) * W);
        const Vec<CPT> r = ld_plain<CPT>(rho + (sa + __ldg(sBt + u)) * W);
        Vec<CPT> v;
#pragma unroll
        for (int k = 0; k < CPT; ++k) v.x[k] = p.x[k] * r.x[k];
        kahan_add<CPT>(acc, comp, v);
      }
    }
  };
  auto output = [&](int64_t t, const Vec<CPT> &val) {
    if (T.kind == TASK_CHILD) {
      const int64_t o = ((int64_t)tile * P.sep_rows + T.dst_row + t) * W + lane * CPT;
      const Vec<CPT> ph = ld_plain<CPT>(A.phistar + o);
      Vec<CPT> r;
#pragma unroll
      for (int k = 0; k < CPT; ++k) r.x[k] = (ph.x[k] > 0.f) ? val.x[k] / ph.x[k] : 0.f;  // 0/0 := 0
      st_plain<CPT>(A.rho + o, r);
    } else {
      st_plain<CPT>(A.post + ((int64_t)tile * P.post_rows + T.dst_row + t) * W + lane * CPT, val);
    }
  };

  if (!it.split) {
    for (int64_t t = it.t0 + warp; t < it.t0 + it.nt; t += kWarps) {
      Vec<CPT> acc = vzero<CPT>(), comp = vzero<CPT>();
      rows(t, 0, T.U, acc, comp);
      output(t, acc);
    }
  } else {
    const int64_t t = it.t0;
    const int64_t q = (it.nu + kWarps - 1) / kWarps;
    const int64_t ua = it.u0 + warp * q;
    const int64_t ub = min(ua + q, it.u0 + it.nu);
    Vec<CPT> acc = vzero<CPT>(), comp = vzero<CPT>();
    if (ua < ub) rows(t, ua, ub, acc, comp);
    st_plain<CPT>(red + warp * W + lane * CPT, acc);
    __syncthreads();
    if (warp == 0) {
      Vec<CPT> tot = vzero<CPT>();
      for (int w = 0; w < kWarps; ++w) {
        const Vec<CPT> x = ld_plain<CPT>(red + w * W + lane * CPT);
#pragma unroll
        for (int k = 0; k < CPT; ++k) tot.x[k] += x.x[k];
      }
      if (it.npieces == 1)
        output(t, tot);
      else
        st_plain<CPT>(A.partial + ((int64_t)tile * P.n_partials + it.partial) * W + lane * CPT, tot);
    }
    if (it.npieces > 1) {
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned old = atomicAdd(&A.counters[(int64_t)tile * P.n_groups + it.group], 1u);
        s_last = (old == (unsigned)(it.npieces - 1));
      }
      __syncthreads();
      if (s_last && warp == 0) {
        __threadfence();
        const int first = it.partial - it.piece;
        Vec<CPT> tot = vzero<CPT>();
        for (int p = 0; p < it.npieces; ++p) {
          const Vec<CPT> x = ld_cg<CPT>(A.partial + ((int64_t)tile * P.n_partials + first + p) * W + lane * CPT);
#pragma unroll
          for (int k = 0; k < CPT; ++k) tot.x[k] += x.x[k];
        }
        output(t, tot);
        if (lane == 0) A.counters[(int64_t)tile * P.n_groups + it.group] = 0u;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// finalize: one warp per case
// ---------------------------------------------------------------------------
__global__ void k_finalize(DevPlan P, DevArena A, int W, int32_t n_cases, int64_t root_sep_row,
                           double *__restrict__ log_pe, double *__restrict__ post,
                           int32_t *__restrict__ status) {
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= n_cases) return;
  const int64_t tile = wid / W;
  const int c = (int)(wid % W);
  // Messages multiplied into a parent were scaled by 2^-k: add k back.
  // Every component root contributes the log of its total -- except a
  // component without any observed variable, whose probability is exactly 1
  // (a sum over all states of a product of CPTs) and contributes 0; its
  // cliques' exponents are left out with it.
  long long K = 0;
  double lz = 0.0;
  int zero = 0;
  for (int cl = lane; cl < P.n_cliques; cl += 32) {
    const DClique &D = P.cl[cl];
    if (!D.is_root) continue;
    bool observed = false;
    for (int k = P.comp_ptr[cl]; k < P.comp_ptr[cl + 1] && !observed; ++k)
      observed = A.ev[(tile * P.n_vars + P.comp_vars[k]) * W + c] >= 0;
    if (!observed) continue;
    const float z = A.phistar[(tile * P.sep_rows + D.sep_row) * W + c];
    if (z > 0.f) lz += log((double)z); else zero = 1;
    K += D.comp_base_exp;
    for (int k = D.comp_begin; k < D.comp_end; ++k)
      K += pow2_exp(A.maxbits[(tile * P.n_cliques + P.comp_cliques[k]) * W + c]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    K += __shfl_xor_sync(0xffffffffu, K, o);
    lz += __shfl_xor_sync(0xffffffffu, lz, o);
    zero |= __shfl_xor_sync(0xffffffffu, zero, o);
  }
  (void)root_sep_row;
  const int bad = A.bad[tile * W + c];
  const int st = bad ? JT_CASE_BAD_EVIDENCE : (zero ? JT_CASE_ZERO_EVIDENCE : JT_CASE_OK);
  if (lane == 0) {
    double lp;
    if (st == JT_CASE_OK)
      lp = lz + (double)K * 0.69314718055994530942;
    else if (st == JT_CASE_ZERO_EVIDENCE)
      lp = -INFINITY;
    else
      lp = NAN;
    log_pe[wid] = lp;
    status[wid] = st;
  }
  double *out = post + wid * P.post_rows;
  for (int v = lane; v < P.n_vars; v += 32) {
    const int64_t off = P.post_off[v];
    const int r = P.card[v];
    const int ev = A.ev[(tile * P.n_vars + v) * W + c];
    if (st != JT_CASE_OK) {
      for (int j = 0; j < r; ++j) out[off + j] = NAN;
    } else if (ev >= 0) {
      for (int j = 0; j < r; ++j) out[off + j] = (j == ev) ? 1.0 : 0.0;
    } else {
      const float *m = A.post + (tile * P.post_rows + off) * W + c;
      double s = 0.0;
      for (int j = 0; j < r; ++j) s += (double)m[(int64_t)j * W];
      for (int j = 0; j < r; ++j) out[off + j] = (double)m[(int64_t)j * W] / s;
    }
  }
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

size_t collect_smem_bytes(int cpt, int max_maps) { return collect_smem_layout(cpt, max_maps, nullptr, nullptr); }

void launch_evidence(int cpt, const int32_t *d_ev_in, int32_t n_cases, const DevPlan &P,
                     const DevArena &A, cudaStream_t s) {
  const int W = 32 * cpt;
  const int64_t total = (int64_t)A.tiles * W * P.n_vars;
  unsigned blocks = (unsigned)std::min<int64_t>(blocks_for(total, 256), 152 * 16);
  k_evidence<<<blocks, 256, 0, s>>>(d_ev_in, n_cases, P, A, W);
}

template <int CPT>
static void collect_t(const DevPlan &P, const DevArena &A, int64_t b, int64_t n, int max_maps, cudaStream_t s) {
  const size_t smem = collect_smem_bytes(CPT, max_maps);
  dim3 grid((unsigned)n, (unsigned)A.tiles);
  k_collect<CPT><<<grid, kThreads, smem, s>>>(P, A, b);
}

cudaError_t configure_collect_smem(int cpt, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  if (cpt == 4) return cudaFuncSetAttribute(k_collect<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (cpt == 2) return cudaFuncSetAttribute(k_collect<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaFuncSetAttribute(k_collect<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

void launch_collect(int cpt, const DevPlan &P, const DevArena &A, int64_t b, int64_t n, int max_maps,
                    cudaStream_t s) {
  if (n <= 0) return;
  if (cpt == 4) collect_t<4>(P, A, b, n, max_maps, s);
  else if (cpt == 2) collect_t<2>(P, A, b, n, max_maps, s);
  else collect_t<1>(P, A, b, n, max_maps, s);
}

void launch_distribute(int cpt, const DevPlan &P, const DevArena &A, int64_t b, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  dim3 grid((unsigned)n, (unsigned)A.tiles);
  if (cpt == 4) k_distribute<4><<<grid, kThreads, 0, s>>>(P, A, b);
  else if (cpt == 2) k_distribute<2><<<grid, kThreads, 0, s>>>(P, A, b);
  else k_distribute<1><<<grid, kThreads, 0, s>>>(P, A, b);
}

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

void launch_finalize(int cpt, const DevPlan &P, const DevArena &A, int32_t n_cases,
                            int64_t root_sep_row, double *d_log_pe, double *d_post, int32_t *d_status,
                            cudaStream_t s) {
  if (n_cases <= 0) return;
  const int W = 32 * cpt;
  const int threads = 256;
  const unsigned blocks = blocks_for((int64_t)n_cases * 32, threads);
  k_finalize<<<blocks, threads, 0, s>>>(P, A, W, n_cases, root_sep_row, d_log_pe, d_post, d_status);
}

}  // namespace jt
