// lem_forest.cuh -- one thread block runs Algs 3-6 of Barnes (arXiv:1803.02977)
// on a set of trees of one grid by itself, with block barriers only.  The
// batched form uses it for the trees of a realization that do not fit a
// warp's queue (lem_tiles.cuh).
//
// The queue lives in global memory in breadth-first order: level 0 (the
// trees' roots, given) first, then each level's donors in the order of their
// receivers, each entry with its donor mask (pqm), receiver code (pqk) and
// the queue position of its receiver (pqf, levels >= 1).  Accumulation runs
// on a queue-ordered count array, each entry adding its final count to its
// receiver's (deepest level first); erosion gathers elevations.  A deep
// forest is latency-bound, level by level, so each level reads as little as
// it can after the previous one: the level offsets are mirrored in shared
// memory (splev, the block's warp slices, idle by then), and a count push
// needs only the entry's own words.
#pragma once

#include "lem_step_kernel.cuh"

namespace lem {

template <int BD, int PI>
struct ForestSmem {
  static constexpr int kW = BD / 32;
  int chunk[PI * kW];
  int chunk_total;
  int wcount[kW];
  int wbase[kW];
};

struct ForestGrid {
  int nx, ny, N;
  float* h;
  uint8_t* code;
  uint8_t* mask;
  int* pq;
  uint8_t* pqm;
  uint8_t* pqk;
  int* pqf;
  int* cntq;
  int* plev;       // level offsets, capacity N + 1
  int* splev;      // their first splev_cap entries, mirrored in shared memory
  int splev_cap;
  float Udt;       // U*dt, rounded once to float
  __device__ __forceinline__ void set_level(int l, int v) const {
    plev[l] = v;
    if (l < splev_cap) splev[l] = v;
  }
  __device__ __forceinline__ int level(int l) const { return l < splev_cap ? splev[l] : plev[l]; }
};

// One round of Alg 3: the entries [base, base + PIR * BD) of the level
// [lo, hi), PIR per thread (strided, so the loads coalesce), emit their
// donors at run.. in parent order.  Returns the number emitted.
template <int BD, int PI, int PIR>
__device__ __forceinline__ int forest_round(const ForestGrid& g, ForestSmem<BD, PI>& s, int lo,
                                            int hi, int base, int run) {
  constexpr int W = BD / 32;
  constexpr int C = PIR * W;          // chunk totals of the round
  constexpr int PER = (C + 31) / 32;  // chunk totals per lane of warp 0
  static_assert(PIR <= PI, "chunk totals fit");
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int nx = g.nx;
  int cs[PIR], ms[PIR];
#pragma unroll
  for (int i = 0; i < PIR; ++i) {
    const int j = base + i * BD + t;
    cs[i] = (j < hi) ? g.pq[j] : -1;
  }
  if (lo == 0) {
#pragma unroll
    for (int i = 0; i < PIR; ++i) ms[i] = (cs[i] >= 0) ? g.pqm[base + i * BD + t] : 0;
  } else {
#pragma unroll
    for (int i = 0; i < PIR; ++i) ms[i] = (cs[i] >= 0) ? g.mask[cs[i]] : 0;
#pragma unroll
    for (int i = 0; i < PIR; ++i)
      if (cs[i] >= 0) g.pqm[base + i * BD + t] = (uint8_t)ms[i];
  }
  int pos_i[PIR];
#pragma unroll
  for (int i = 0; i < PIR; ++i) {
    const int cnt = __popc(ms[i]);
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    pos_i[i] = x - cnt;
    if (lane == 31) s.chunk[i * W + w] = x;
  }
  __syncthreads();
  if (w == 0) {
    int v[PER], sum = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = lane * PER + q;
      v[q] = (idx < C) ? s.chunk[idx] : 0;
      sum += v[q];
    }
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s.chunk_total = x;
    int acc = x - sum;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = lane * PER + q;
      if (idx < C) s.chunk[idx] = acc;
      acc += v[q];
    }
  }
  __syncthreads();
  const int tot = s.chunk_total;
#pragma unroll
  for (int i = 0; i < PIR; ++i) pos_i[i] += run + s.chunk[i * W + w];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PIR; ++i) {
    int pos = pos_i[i];
    const int parent = base + i * BD + t;
    int msk = ms[i];
    while (msk) {
      const int k = __ffs(msk) - 1;
      msk &= msk - 1;
      g.pq[pos] = cs[i] + nbr_off(k, nx);
      g.pqk[pos] = (uint8_t)(7 - k);
      g.pqf[pos] = parent;
      g.cntq[pos] = 1;
      ++pos;
    }
  }
  return tot;
}

// Alg 3: expand levels from level 0 = [0, n0) (pq with pqm and pqk filled).
// A level of at most BD entries (deep trees are mostly such levels) takes one
// round of one entry per thread; wider ones rounds of PI per thread.
// Returns the number of levels PL; the level offsets go to plev (and splev).
template <int BD, int PI>
__device__ int forest_levels(const ForestGrid& g, int n0, ForestSmem<BD, PI>& s) {
  const int t = threadIdx.x;
  int lo = 0, hi = n0, PL = 1;
  if (t == 0) {
    g.set_level(0, 0);
    g.set_level(1, n0);
  }
  while (lo < hi) {
    int run = hi;
    if (hi - lo <= BD) {
      run += forest_round<BD, PI, 1>(g, s, lo, hi, lo, run);
    } else {
      for (int base = lo; base < hi; base += PI * BD)
        run += forest_round<BD, PI, PI>(g, s, lo, hi, base, run);
    }
    __syncthreads();
    if (run == hi) break;
    ++PL;
    if (t == 0) g.set_level(PL, run);
    lo = hi;
    hi = run;
  }
  __syncthreads();
  return PL;
}

// Alg 4, levels PL-1 down to 2: every entry adds its count (1 when it was
// queued, final once its own level comes up) to its receiver's entry; level
// 1 feeds only level 0, which does not erode.
template <int BD>
__device__ void forest_accumulate(const ForestGrid& g, int PL) {
  const int t = threadIdx.x;
  for (int l = PL - 1; l >= 2; --l) {
    const int l0 = g.level(l), l1 = g.level(l + 1);
    for (int j = l0 + t; j < l1; j += BD) atomicAdd(g.cntq + g.pqf[j], g.cntq[j]);
    __syncthreads();
  }
}

// g = F/(1+F) for this grid's parameters; small counts come from a
// shared-memory table built per realization.
struct ErosionFactors {
  const float* tab;  // [0,TN) cardinal, [TN,2TN) diagonal
  int TN;
  double Kdt, m, dx, dxd, area;
  __device__ float operator()(int count, bool diag) const {
    if (count < TN) return tab[(diag ? TN : 0) + count];
    const double A = (double)count * area;
    const double F = Kdt * pow(A, m) / (diag ? dxd : dx);
    return (float)(F / (1.0 + F));
  }
};

// Algs 5-6 (FP32 increment form): uplift level-0 pits, then levels 1 up.
template <int BD>
__device__ void forest_erode(const ForestGrid& g, int PL, const ErosionFactors& ef) {
  const int t = threadIdx.x;
  const int n0 = g.plev[1];
  for (int j = t; j < n0; j += BD)
    if (g.pqk[j] == kSink) {
      const int c = g.pq[j];
      g.h[c] = __fadd_rn(g.h[c], g.Udt);
    }
  __syncthreads();
  for (int l = 1; l < PL; ++l) {
    const int l0 = g.level(l), l1 = g.level(l + 1);
    for (int j = l0 + t; j < l1; j += BD) {
      const int c = g.pq[j], k = g.pqk[j];
      const float gk = ef(g.cntq[j], nbr_diag(k));
      const float h0 = __fadd_rn(g.h[c], g.Udt);
      const float hr = g.h[c + nbr_off(k, g.nx)];
      g.h[c] = __fmaf_rn(-gk, __fsub_rn(h0, hr), h0);
    }
    __syncthreads();
  }
}

}  // namespace lem
