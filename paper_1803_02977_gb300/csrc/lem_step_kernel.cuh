// lem_step_kernel.cuh -- the persistent cooperative kernel that runs the
// per-timestep method of Barnes (arXiv:1803.02977), Section "The Algorithm",
// Algorithms 1-6, on one GB300.
//
// One launch covers any subset of the stages (phase bits) for nsteps steps.
// Stages are separated by device-wide barriers (grid_barrier); breadth-first
// levels are processed one barrier apart ("for-parallel" loops of the
// paper), except that a run of narrow levels (at most kNarrow cells each) is
// processed by block 0 alone with block-local barriers while the other blocks
// wait once (the paper's barrier elimination, Section "On Parallelism").
//
// Data layout (all in HBM, row-major grid order unless stated):
//   h      elevations (double or float), caller owned, updated in place
//   code   u8  receiver code per cell (0..7 neighbour k, 8 none)
//   mask   u8  donor mask per cell: bit k set <=> neighbour k drains here
//   queue  i32 cells in breadth-first order (Alg 3's Queue)
//   levels i32 level offsets into queue (Alg 3's Levels), L+1 used
//   cnt    i32 or i64 cell counts (Alg 4's A in units of cells)
#pragma once

#include "lem_device.cuh"

namespace lem {

template <typename HT, typename CT>
struct StepArgs {
  int nx, ny, N;
  HT* h;
  const double* Uf;     // optional per-cell uplift rate
  double U, dt;         // scalar uplift rate, time step
  double Kdt;           // K*dt
  double m, dx, dxd;    // area exponent, cardinal and diagonal distance
  double area_scale;
  uint8_t* code;
  uint8_t* mask;
  int* queue;
  int* levels;
  CT* cnt;
  const double* Ftab;   // F for counts < kTableN: [0,N) cardinal, [N,2N) diagonal
  const float* gtab;    // F/(1+F) rounded to float, same layout
  DevState* st;
  int* partial;         // one int per block
  int phases;
  int nsteps;
  int frozen;           // receivers frozen: codes are inputs, not recomputed
};

constexpr int kBD = 512;           // threads per block of the persistent kernel
constexpr int kNarrow = 2 * kBD;   // a level this small is run by block 0 alone

// Alg 1 for one interior cell: steepest strictly positive descent, slope
// compared as (h_c - h_n) * w in FP64 (w = 1 or 1/sqrt(2)), strict '>'
// against an initial maximum of zero, so the lowest k wins ties.
template <typename HT>
__device__ __forceinline__ int receiver_code(const HT* __restrict__ h, int c, int nx) {
  const double hc = (double)h[c];
  double smax = 0.0;
  int best = kSink;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double hn = (double)h[c + nbr_off(k, nx)];
    const double d = __dsub_rn(hc, hn);
    const double s = nbr_diag(k) ? __dmul_rn(d, kInvSqrt2) : d;
    if (s > smax) {
      smax = s;
      best = k;
    }
  }
  return best;
}

// Alg 2 for one cell (perimeter included): bit k set iff neighbour k is in
// the grid and its receiver code points back at this cell (code 7-k).
__device__ __forceinline__ int donor_mask(const uint8_t* __restrict__ code, int c, int x, int y,
                                          int nx, int ny) {
  int msk = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int xn = x + nbr_dx(k), yn = y + nbr_dy(k);
    if (xn >= 0 && yn >= 0 && xn < nx && yn < ny) {
      if (code[c + nbr_off(k, nx)] == 7 - k) msk |= 1 << k;
    }
  }
  return msk;
}

template <typename HT, typename CT>
__device__ __forceinline__ double erosion_F(const StepArgs<HT, CT>& a, CT count, bool diag) {
  if (count < (CT)kTableN) return a.Ftab[(diag ? kTableN : 0) + (int)count];
  const double A = __dmul_rn((double)count, a.area_scale);
  return __ddiv_rn(__dmul_rn(a.Kdt, pow(A, a.m)), diag ? a.dxd : a.dx);
}

template <typename HT, typename CT>
__device__ __forceinline__ double uplift_dt(const StepArgs<HT, CT>& a, int c) {
  return a.Uf ? __dmul_rn(a.Uf[c], a.dt) : __dmul_rn(a.U, a.dt);
}

// Alg 5 for a cell without receiver: uplift if interior.
template <typename HT, typename CT>
__device__ __forceinline__ void uplift_sink(const StepArgs<HT, CT>& a, int c) {
  const int x = c % a.nx, y = c / a.nx;
  if (x == 0 || y == 0 || x == a.nx - 1 || y == a.ny - 1) return;
  if constexpr (sizeof(HT) == 8) {
    a.h[c] = __dadd_rn(a.h[c], uplift_dt(a, c));
  } else {
    a.h[c] = __fadd_rn(a.h[c], (float)uplift_dt(a, c));
  }
}

// Alg 5 + Alg 6 (n = 1) for one cell of level >= 1.
template <typename HT, typename CT>
__device__ __forceinline__ void erode_cell(const StepArgs<HT, CT>& a, int c) {
  const int k = a.code[c];
  const int r = c + nbr_off(k, a.nx);
  const CT count = a.cnt[c];
  if constexpr (sizeof(HT) == 8) {
    const double F = erosion_F(a, count, nbr_diag(k));
    const double h0 = __dadd_rn(a.h[c], uplift_dt(a, c));
    const double num = __dadd_rn(h0, __dmul_rn(F, a.h[r]));
    a.h[c] = __ddiv_rn(num, __dadd_rn(1.0, F));
  } else {
    float g;
    if (count < (CT)kTableN) {
      g = a.gtab[(nbr_diag(k) ? kTableN : 0) + (int)count];
    } else {
      const double F = erosion_F(a, count, nbr_diag(k));
      g = (float)(F / (1.0 + F));
    }
    const float h0 = __fadd_rn(a.h[c], (float)uplift_dt(a, c));
    const float hr = a.h[r];
    a.h[c] = __fmaf_rn(-g, __fsub_rn(h0, hr), h0);
  }
}

// Alg 4 for one cell: 1 + the donors' counts.
template <typename HT, typename CT>
__device__ __forceinline__ void accumulate_cell(const StepArgs<HT, CT>& a, int c) {
  int msk = a.mask[c];
  CT s = 1;
  while (msk) {
    const int k = __ffs(msk) - 1;
    msk &= msk - 1;
    s += a.cnt[c + nbr_off(k, a.nx)];
  }
  a.cnt[c] = s;
}

// Emit the donors of `c` (mask msk) at queue[pos...], k order.
__device__ __forceinline__ void emit_donors(int* __restrict__ queue, int pos, int c, int msk,
                                            int nx) {
  while (msk) {
    const int k = __ffs(msk) - 1;
    msk &= msk - 1;
    queue[pos++] = c + nbr_off(k, nx);
  }
}

template <typename HT, typename CT>
__global__ void __launch_bounds__(kBD, 2) lem_step_kernel(StepArgs<HT, CT> a) {
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, t = threadIdx.x;
  const int gtid = b * kBD + t, gstride = (int)G * kBD;
  const int nx = a.nx, ny = a.ny, N = a.N;
  __shared__ int s_scan[kBD / 32];
  __shared__ long long s_sum[kBD / 32];

  for (int step = 0; step < a.nsteps; ++step) {
    int L_here = -1;  // L found by this launch's Alg 3 phase
    // ---- Alg 1 receivers, Alg 2 donor masks, level 0 of Alg 3 ------------
    if (a.phases & kPhRec) {
      if (!a.frozen) {
        for (int c = gtid; c < N; c += gstride) {
          const int x = c % nx, y = c / nx;
          const bool perim = (x == 0 || y == 0 || x == nx - 1 || y == ny - 1);
          a.code[c] = (uint8_t)(perim ? kSink : receiver_code(a.h, c, nx));
        }
        if (!grid_barrier(a.st, G)) return;
      }
      // Each block owns one contiguous chunk: donor masks, then the sinks of
      // the chunk in ascending address order.
      const int chunk = (N + (int)G - 1) / (int)G;
      const int c0 = min(N, b * chunk), c1 = min(N, c0 + chunk);
      long long nsink = 0;
      for (int c = c0 + t; c < c1; c += kBD) {
        const int x = c % nx, y = c / nx;
        a.mask[c] = (uint8_t)donor_mask(a.code, c, x, y, nx, ny);
        nsink += (a.code[c] == kSink);
      }
      nsink = block_sum<kBD>(nsink, s_sum);
      if (t == 0) a.partial[b] = (int)nsink;
      if (!grid_barrier(a.st, G)) return;
      int prefix = 0, total = 0;
      for (int i = t; i < (int)G; i += kBD) {
        const int v = a.partial[i];
        total += v;
        if (i < b) prefix += v;
      }
      prefix = (int)block_sum<kBD>(prefix, s_sum);
      total = (int)block_sum<kBD>(total, s_sum);
      int run = prefix;
      for (int base = c0; base < c1; base += kBD) {
        const int c = base + t;
        const int f = (c < c1) && (a.code[c] == kSink);
        int tot;
        const int ex = block_exclusive_scan<kBD>(f, &tot, s_scan);
        if (f) a.queue[run + ex] = c;
        run += tot;
      }
      if (b == 0 && t == 0) {
        a.levels[0] = 0;
        a.levels[1] = total;
      }
      if (!grid_barrier(a.st, G)) return;
    }

    // ---- Alg 3: breadth-first levels -------------------------------------
    if (a.phases & kPhLev) {
      int lo = 0, hi = a.levels[1], l = 0;
      while (true) {
        const int S = hi - lo;
        if (S <= kNarrow) {
          if (b == 0) {
            // block 0 alone: consecutive narrow levels, block barriers only
            bool done = false;
            while (true) {
              int run = hi;
              for (int base = lo; base < hi; base += kBD) {
                const int j = base + t;
                int c = 0, msk = 0;
                if (j < hi) {
                  c = a.queue[j];
                  msk = a.mask[c];
                }
                int tot;
                const int ex = block_exclusive_scan<kBD>(__popc(msk), &tot, s_scan);
                if (msk) emit_donors(a.queue, run + ex, c, msk, nx);
                run += tot;
              }
              __syncthreads();
              if (t == 0) a.levels[l + 2] = run;
              if (run == hi) {
                done = true;
                break;
              }
              lo = hi;
              hi = run;
              ++l;
              if (hi - lo > kNarrow) break;
            }
            if (t == 0) {
              a.st->bfs_lo = lo;
              a.st->bfs_hi = hi;
              a.st->bfs_level = l;
              a.st->bfs_done = done ? 1 : 0;
            }
          }
          if (!grid_barrier(a.st, G)) return;
          lo = ld_volatile(&a.st->bfs_lo);
          hi = ld_volatile(&a.st->bfs_hi);
          l = ld_volatile(&a.st->bfs_level);
          if (ld_volatile(&a.st->bfs_done)) break;
          continue;
        }
        // wide level: count, barrier, deterministic offsets, write, barrier
        const int chunk = (S + (int)G - 1) / (int)G;
        const int j0 = min(hi, lo + b * chunk), j1 = min(hi, j0 + chunk);
        long long nd = 0;
        for (int j = j0 + t; j < j1; j += kBD) nd += __popc(a.mask[a.queue[j]]);
        nd = block_sum<kBD>(nd, s_sum);
        if (t == 0) a.partial[b] = (int)nd;
        if (!grid_barrier(a.st, G)) return;
        int prefix = 0, total = 0;
        for (int i = t; i < (int)G; i += kBD) {
          const int v = a.partial[i];
          total += v;
          if (i < b) prefix += v;
        }
        prefix = (int)block_sum<kBD>(prefix, s_sum);
        total = (int)block_sum<kBD>(total, s_sum);
        int run = hi + prefix;
        for (int base = j0; base < j1; base += kBD) {
          const int j = base + t;
          int c = 0, msk = 0;
          if (j < j1) {
            c = a.queue[j];
            msk = a.mask[c];
          }
          int tot;
          const int ex = block_exclusive_scan<kBD>(__popc(msk), &tot, s_scan);
          if (msk) emit_donors(a.queue, run + ex, c, msk, nx);
          run += tot;
        }
        if (b == 0 && t == 0) a.levels[l + 2] = hi + total;
        if (!grid_barrier(a.st, G)) return;
        if (total == 0) break;
        lo = hi;
        hi = hi + total;
        ++l;
      }
      // L = l + 1 levels; every cell must have been reached
      const int L = l + 1;
      L_here = L;
      if (b == 0 && t == 0) a.st->nlevels = L;
      if (a.levels[L] != N) {
        if (b == 0 && t == 0) set_error(a.st, kErrInval);
        return;
      }
    }

    const int L = L_here >= 0 ? L_here : ld_volatile(&a.st->nlevels);

    // ---- Alg 4: accumulation, highest level down --------------------------
    if (a.phases & kPhAcc) {
      int l = L - 1;
      while (l >= 0) {
        int lo = a.levels[l], hi = a.levels[l + 1];
        if (hi - lo <= kNarrow) {
          int ll = l;
          if (b == 0) {
            while (ll >= 0) {
              lo = a.levels[ll];
              hi = a.levels[ll + 1];
              if (hi - lo > kNarrow) break;
              for (int j = lo + t; j < hi; j += kBD) accumulate_cell(a, a.queue[j]);
              __syncthreads();
              --ll;
            }
          } else {
            while (ll >= 0 && a.levels[ll + 1] - a.levels[ll] <= kNarrow) --ll;
          }
          if (!grid_barrier(a.st, G)) return;
          l = ll;
          continue;
        }
        for (int j = lo + gtid; j < hi; j += gstride) accumulate_cell(a, a.queue[j]);
        if (!grid_barrier(a.st, G)) return;
        --l;
      }
    }

    // ---- Alg 5 + Alg 6: uplift and erosion, level 1 upward ------------------
    if (a.phases & kPhEro) {
      for (int j = gtid; j < a.levels[1]; j += gstride) uplift_sink(a, a.queue[j]);
      if (!grid_barrier(a.st, G)) return;
      int l = 1;
      while (l < L) {
        int lo = a.levels[l], hi = a.levels[l + 1];
        if (hi - lo <= kNarrow) {
          int ll = l;
          if (b == 0) {
            while (ll < L) {
              lo = a.levels[ll];
              hi = a.levels[ll + 1];
              if (hi - lo > kNarrow) break;
              for (int j = lo + t; j < hi; j += kBD) erode_cell(a, a.queue[j]);
              __syncthreads();
              ++ll;
            }
          } else {
            while (ll < L && a.levels[ll + 1] - a.levels[ll] <= kNarrow) ++ll;
          }
          if (!grid_barrier(a.st, G)) return;
          l = ll;
          continue;
        }
        for (int j = lo + gtid; j < hi; j += gstride) erode_cell(a, a.queue[j]);
        if (!grid_barrier(a.st, G)) return;
        ++l;
      }
    }
  }
}

}  // namespace lem
