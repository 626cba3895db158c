// lem_mfd.cu -- flow accumulation with multiple flow directions (Section
// "Multiple Flow Directions"; Eq. 2 with a general split alpha and source w).
//
// Receivers of an interior cell are all its strictly lower neighbours;
// perimeter cells and pits have none.  Cell d sends the fraction
//     alpha(d -> n_k) = s_k^p / sum over its receivers of s^p,
// s_k = (h_d - h_n_k) * w_k with the weights of Alg 1 (1 cardinal, the double
// nearest 1/sqrt2 diagonal), the sum taken in k order.  Eq. 2 then reads
//     A(c) = w(c) + sum over the donors d of c, in k order, of alpha(d -> c) A(d).
// A cell can be computed once all its donors are (the paper's figure on
// multiple flow directions), so the levels are Kahn's order on the donor
// graph: level 0 holds the cells without donors, and a cell joins the level
// after the one of its last donor.  Each cell pulls from its donors in k
// order with separately rounded FP64 operations, so A does not depend on the
// order of the cells within a level: for p = 1 (no power) it matches a serial
// evaluation bit for bit.
//
// One cooperative launch: a pass over every cell (donor counts, the
// receivers' sum of s^p, level 0), then the levels with one grid barrier per
// wide level and runs of narrow levels in block 0.  A frontier cell that
// releases a receiver's last pending donor appends it to the next level
// (warp-aggregated atomics).
#include <cuda_runtime.h>

#include <cstddef>

#include "lem.h"
#include "lem_context.cuh"

namespace lem {

constexpr int kMfdBD = 512;          // threads per block
constexpr int kMfdNarrow = kMfdBD;   // a level this small runs in block 0

struct MfdState {
  int tail;       // entries appended to the queue so far
  int lo, hi;     // the level block 0 hands over
  int done;       // block 0 found the last level
  int nlevels;
};

template <typename HT>
struct MfdArgs {
  int nx, ny;
  const HT* h;
  const double* w;  // per-cell source, or null for 1
  double p;
  double* A;        // out
  int* pending;     // donors not yet computed
  double* norm;     // sum of s^p over the receivers
  int* queue;       // the levels, one after another
  MfdState* ms;
  DevState* st;
};

__device__ __forceinline__ bool mfd_perim(int x, int y, int nx, int ny) {
  return x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
}

// slope weight of neighbour k: the (rounded) difference, scaled for diagonals
__device__ __forceinline__ double mfd_slope(double hi, double lo, int k) {
  const double d = __dsub_rn(hi, lo);
  return nbr_diag(k) ? __dmul_rn(d, kInvSqrt2) : d;
}

// s^p for a positive slope s, as 2^(p log2 s): two FP64 library calls
// instead of the costlier general power, within a few units in the last
// place of it for the slopes of a grid (|p log2 s| well below 2^10)
__device__ __forceinline__ double mfd_pow(double s, double p) {
  return p == 1.0 ? s : exp2(p * log2(s));
}

// Append the lanes' flagged cells to the queue (one atomic per warp).
__device__ __forceinline__ void mfd_append(int* queue, int* tail, bool f, int c) {
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (bal == 0) return;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0) base = atomicAdd(tail, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (f) queue[base + __popc(bal & ((1u << lane) - 1u))] = c;
}

// Eq. 2 for cell c (all donors final), then release its receivers; the
// whole warp calls this (c < 0: an idle lane).
template <typename HT>
__device__ __forceinline__ void mfd_cell(const MfdArgs<HT>& a, int c) {
  const int nx = a.nx, ny = a.ny;
  const bool on = c >= 0;
  int x = 0, y = 0;
  double hc = 0.0;
  if (on) {
    y = c / nx;
    x = c - y * nx;
    hc = (double)a.h[c];
    double acc = a.w ? a.w[c] : 1.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int xn = x + nbr_dx(k), yn = y + nbr_dy(k);
      if (xn < 0 || yn < 0 || xn >= nx || yn >= ny || mfd_perim(xn, yn, nx, ny)) continue;
      const int d = yn * nx + xn;
      const double hd = (double)a.h[d];
      if (!(hd > hc)) continue;
      // c is neighbour 7-k of its donor d
      const double alpha = __ddiv_rn(mfd_pow(mfd_slope(hd, hc, 7 - k), a.p), a.norm[d]);
      acc = __dadd_rn(acc, __dmul_rn(alpha, __ldcg(a.A + d)));
    }
    a.A[c] = acc;
  }
  const bool interior = on && !mfd_perim(x, y, nx, ny);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    bool rel = false;
    int r = 0;
    if (interior) {
      r = c + nbr_off(k, nx);
      if ((double)a.h[r] < hc) rel = atomicSub(&a.pending[r], 1) == 1;
    }
    mfd_append(a.queue, &a.ms->tail, rel, r);
  }
}

template <typename HT>
__global__ void __launch_bounds__(kMfdBD) mfd_kernel(const __grid_constant__ MfdArgs<HT> a) {
  const int nx = a.nx, ny = a.ny;
  const int N = nx * ny;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, t = threadIdx.x;
  const int gtid = b * kMfdBD + t, gstride = (int)G * kMfdBD;
  // donor counts, the receivers' sum of s^p, and level 0 (appended by warps
  // of whole cells: the loop bound is rounded up to the warp)
  const int span = ((N + 31) / 32) * 32;
  for (int c0 = gtid; c0 < ((span + gstride - 1) / gstride) * gstride; c0 += gstride) {
    const int c = c0 < N ? c0 : -1;
    int nd = 0;
    if (c >= 0) {
      const int y = c / nx, x = c - y * nx;
      const double hc = (double)a.h[c];
      const bool interior = !mfd_perim(x, y, nx, ny);
      double sum = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int xn = x + nbr_dx(k), yn = y + nbr_dy(k);
        if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
        const double hn = (double)a.h[yn * nx + xn];
        if (hn > hc && !mfd_perim(xn, yn, nx, ny)) ++nd;
        if (interior && hn < hc) sum = __dadd_rn(sum, mfd_pow(mfd_slope(hc, hn, k), a.p));
      }
      a.pending[c] = nd;
      a.norm[c] = sum;
    }
    mfd_append(a.queue, &a.ms->tail, c >= 0 && nd == 0, c);
  }
  if (!grid_barrier(a.st, G)) return;
  int lo = 0, hi = ld_volatile(&a.ms->tail), l = 0;
  while (lo < hi) {
    if (hi - lo <= kMfdNarrow) {
      // block 0 alone runs consecutive narrow levels with block barriers
      if (b == 0) {
        bool done = false;
        while (true) {
          for (int j0 = lo; j0 < hi; j0 += kMfdBD) {
            const int j = j0 + t;
            mfd_cell(a, j < hi ? __ldcg(a.queue + j) : -1);
          }
          __syncthreads();
          const int nh = ld_volatile(&a.ms->tail);
          __syncthreads();  // every thread has read the tail
          ++l;
          lo = hi;
          hi = nh;
          if (lo == hi) {
            done = true;
            break;
          }
          if (hi - lo > kMfdNarrow) break;
        }
        if (t == 0) {
          a.ms->lo = lo;
          a.ms->hi = hi;
          a.ms->done = done ? 1 : 0;
          a.ms->nlevels = l;
        }
      }
      if (!grid_barrier(a.st, G)) return;
      if (ld_volatile(&a.ms->done)) break;
      lo = ld_volatile(&a.ms->lo);
      hi = ld_volatile(&a.ms->hi);
      l = ld_volatile(&a.ms->nlevels);
      continue;
    }
    // a wide level: every block takes a share, warps of whole lanes
    const int S = hi - lo;
    for (int j0 = gtid - (gtid & 31); j0 < ((S + 31) / 32) * 32; j0 += gstride) {
      const int j = j0 + (t & 31);
      mfd_cell(a, j < S ? __ldcg(a.queue + lo + j) : -1);
    }
    if (!grid_barrier(a.st, G)) return;
    ++l;
    lo = hi;
    hi = ld_volatile(&a.ms->tail);
  }
  if (b == 0 && t == 0) {
    a.ms->nlevels = l;
    if (ld_volatile(&a.ms->tail) != N) set_error(a.st, kErrInval);  // cannot happen
  }
}

template <typename HT>
int mfd_launch_typed(lem_ctx* c, double p, const double* w, double* A) {
  cudaError_t e = cudaSuccess;
  if (!c->mfd_pending) {
    int nsm = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)&mfd_kernel<HT>,
                                                        kMfdBD, 0);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) c->mfd_grid = nsm * (per_sm < 2 ? per_sm : 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->mfd_pending, (size_t)c->N * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->mfd_norm, (size_t)c->N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->mfd_queue, (size_t)c->N * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->mfd_state, sizeof(MfdState));
    if (e != cudaSuccess) {
      cudaFree(c->mfd_pending);
      cudaFree(c->mfd_norm);
      cudaFree(c->mfd_queue);
      cudaFree(c->mfd_state);
      c->mfd_pending = nullptr;
      c->mfd_norm = nullptr;
      c->mfd_queue = nullptr;
      c->mfd_state = nullptr;
      return e == cudaErrorMemoryAllocation ? LEM_ENOMEM : LEM_ECUDA;
    }
  }
  e = cudaMemsetAsync(c->mfd_state, 0, sizeof(MfdState), c->stream);
  MfdArgs<HT> a;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.h = (const HT*)c->h;
  a.w = w;
  a.p = p;
  a.A = A;
  a.pending = c->mfd_pending;
  a.norm = c->mfd_norm;
  a.queue = c->mfd_queue;
  a.ms = (MfdState*)c->mfd_state;
  a.st = c->st;
  void* args[] = {&a};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)&mfd_kernel<HT>, dim3(c->mfd_grid), dim3(kMfdBD),
                                    args, 0, c->stream);
  if (e == cudaSuccess) return LEM_OK;
  return e == cudaErrorMemoryAllocation ? LEM_ENOMEM : LEM_ECUDA;
}

}  // namespace lem

extern "C" {

int lem_accumulate_mfd(lem_ctx* c, double p, const double* dev_w, double* dev_A,
                       int64_t* nlevels) {
  if (!c || !dev_A || !(p > 0.0) || !(p < 1e300)) return LEM_EINVAL;
  if (!c->h) return LEM_ESTATE;
  const int rc = c->p.dtype == LEM_F64 ? lem::mfd_launch_typed<double>(c, p, dev_w, dev_A)
                                       : lem::mfd_launch_typed<float>(c, p, dev_w, dev_A);
  if (rc != LEM_OK) return rc;
  const int s = lem_sync(c);
  if (s != LEM_OK) return s;
  if (nlevels) {
    int L = 0;
    if (cudaMemcpy(&L, (char*)c->mfd_state + offsetof(lem::MfdState, nlevels), sizeof(int),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return LEM_ECUDA;
    *nlevels = L;
  }
  return LEM_OK;
}

}  // extern "C"
