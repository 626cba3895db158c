// lem_adjoint.cu -- reverse-mode derivative of the n-hat = 1 time step of
// Barnes (arXiv:1803.02977), Alg 5 + Alg 6, over each step's frozen receiver
// graph (the graph is piecewise constant in the elevations, so its derivative
// is zero almost everywhere).  The paper has no adjoint; this serves the
// inverse problems its introduction motivates.
//
// One step maps h to h' with, for an eroding cell c of receiver r,
//   (1+F_c) h'_c = h_c + dt U_c + F_c h'_r,   F_c = K dt A_c^m / d_c,
// h'_c = h_c + dt U_c for interior pits and h'_c = h_c on the perimeter.
// Given lambda = dL/dh', let mu_c be the total adjoint of h'_c.  Because h'_d
// of each donor d depends on h'_c with weight g_d = F_d/(1+F_d),
//   mu_c = lambda_c + sum over donors d of c of mu_d g_d     (donors first),
// and then, for eroding cells,
//   dL/dh_c = mu_c/(1+F_c),  dL/dU_c += dt mu_c/(1+F_c),
//   dL/dK   += mu_c (h'_r - h'_c)/(1+F_c) * dF_c/dK,  dF_c/dK = dt A_c^m / d_c;
// pits pass mu_c to dL/dh_c and dt*mu_c to dL/dU_c; the perimeter passes mu_c.
// One cooperative launch per step of the sweep: Algs 1-2 on the step's input
// elevations (its frozen graph), then each warp takes tiles and, for the
// trees rooted in its tile, rebuilds their breadth-first queue in shared
// memory (as the forward warp tier does), accumulates counts and sweeps mu
// from the deepest level up, each entry pulling its donors in k order.  If a
// tile's trees do not fit, the same launch redoes the step on device-wide
// levels.  Every cell's outputs of the step (dL/dh, and its dL/dU and dL/dK
// terms) are written, not accumulated, so either form can produce them; the
// terms are then added to per-cell running sums, and dL/dK is reduced over
// the cells in a fixed order at the end, so the result does not depend on
// how work was spread over blocks.
#include <cmath>
#include <cstring>
#include <vector>

#include "lem.h"
#include "lem_context.cuh"

using namespace lem;

namespace {

// One step of the sweep: the step maps elevations s.h (its input) to hnext.
struct AdjArgs {
  StepArgs<double, int> s;  // grid, input elevations, codes, masks, queues, tables, state
  const double2* Gtab;      // {dF/dK cardinal, dF/dK diagonal} by count
  const double* hnext;      // the step's output elevations
  const double* lam;        // dL/dh' of the output
  double* lam_prev;         // dL/dh of the input (written for every cell)
  double* gU;               // this step's dL/dU term per cell (written)
  double* gK;               // this step's dL/dK term per cell (written)
  double* dLdU;             // running dL/dU
  double* dK_cell;          // running dL/dK term per cell
  double* mu;               // device-wide form: mu per cell
};

// g = F/(1+F) and dF/dK for a cell of `count` cells and diagonal flag diag.
__device__ __forceinline__ void factors(const AdjArgs& a, int count, bool diag, double* g,
                                        double* G) {
  if (count < kTableN) {
    *g = a.s.Ftab[(diag ? kTableN : 0) + count].y;
    const double2 gg = a.Gtab[count];
    *G = diag ? gg.y : gg.x;
    return;
  }
  const double Am = pow((double)count * a.s.area_scale, a.s.m);
  const double d = diag ? a.s.dxd : a.s.dx;
  const double F = a.s.Kdt * Am / d;
  *g = F / (1.0 + F);
  *G = a.s.dt * Am / d;
}

// The step's outputs for cell c of receiver code k, count and total adjoint mu.
__device__ __forceinline__ void cell_outputs(const AdjArgs& a, int c, int k, int count, double mu) {
  if (k == kEdge) {
    a.lam_prev[c] = mu;
    a.gU[c] = 0.0;
    a.gK[c] = 0.0;
  } else if (k == kSink) {
    a.lam_prev[c] = mu;
    a.gU[c] = a.s.dt * mu;
    a.gK[c] = 0.0;
  } else {
    double g, Gc;
    factors(a, count, nbr_diag(k), &g, &Gc);
    const double w = mu * (1.0 - g);  // mu / (1 + F)
    a.lam_prev[c] = w;
    a.gU[c] = a.s.dt * w;
    a.gK[c] = w * (a.hnext[c + nbr_off(k, a.s.nx)] - a.hnext[c]) * Gc;
  }
}

// The sweep's tiles are 32 x kAdjTileH cells: smaller than the forward
// step's, so that a tile's trees (with the larger entries below) rarely
// outgrow a warp's slice.
constexpr int kAdjTileH = 4;

// A warp's queue for the sweep: entry j has cell c[j], pd[j] = count << 16 |
// parent << 4 | receiver code (as the forward warp tier), fd[j] = position
// of its first donor << 4 | number of donors, and v[j]: dL/dh' of the cell,
// copied in when the entry is created, then its total adjoint mu.
struct AdjTileQ {
  static constexpr int kHead = kTileLvBytes;
  static constexpr int kCap = ((kWarpBytes - kHead) / (8 + 4 + 4 + 2)) & ~7;
  static_assert(kCap >= kTileW * kAdjTileH, "a tile's level 0 always fits");
  static_assert(kCap < (1 << 12), "first donor position fits fd");
  unsigned short* lev;
  double* v;
  int* c;
  unsigned* pd;
  unsigned short* fd;
  __device__ __forceinline__ explicit AdjTileQ(unsigned char* base) {
    lev = reinterpret_cast<unsigned short*>(base);
    v = reinterpret_cast<double*>(base + kHead);
    c = reinterpret_cast<int*>(base + kHead + 8 * kCap);
    pd = reinterpret_cast<unsigned*>(base + kHead + 12 * kCap);
    fd = reinterpret_cast<unsigned short*>(base + kHead + 16 * kCap);
  }
};

// The sweep of the trees rooted in `tile`, by one warp.  Returns the number
// of cells handled, or -1 if they do not fit (nothing was written).
__device__ __forceinline__ int tile_adjoint(const AdjArgs& a, const AdjTileQ& q, const int* off,
                                            int tile, int lane) {
  constexpr int TH = kAdjTileH;
  const int nx = a.s.nx, ny = a.s.ny, tiles_x = a.s.tiles_x;
  const unsigned lt = (1u << lane) - 1u;
  const uint8_t* const mask = a.s.mask;
  const uint8_t* const code = a.s.code;
  const double* const lam = a.lam;
  int n = 0;
  {
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int x = tx * kTileW + lane, y0 = ty * TH;
    int cd[TH];
#pragma unroll
    for (int r = 0; r < TH; ++r) {
      const int y = y0 + r;
      cd[r] = (x < nx && y < ny) ? code[(size_t)y * nx + x] : 0;
    }
#pragma unroll
    for (int r = 0; r < TH; ++r) {
      const bool f = cd[r] >= kSink;
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (f) {
        const int pos = n + __popc(bal & lt);
        const int c = (y0 + r) * nx + x;
        q.c[pos] = c;
        q.pd[pos] = (unsigned)cd[r];
        cp_async_elem(q.v + pos, lam + c, true);
      }
      n += __popc(bal);
    }
  }
  if (lane == 0) {
    q.lev[0] = 0;
    q.lev[1] = (unsigned short)n;
  }
  __syncwarp();
  // Alg 3 as in the forward warp tier (first-in first-out windows), also
  // recording where each entry's donors start
  int head = 0, tail = n, L = 1, B = n;
  while (head < tail) {
    const int w = min(32, tail - head);
    const int j = head + lane;
    int c = 0, msk = 0;
    if (lane < w) {
      c = q.c[j];
      msk = mask[c];
    }
    const int k = __popc(msk);
    int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    if (tail + tot > AdjTileQ::kCap) {
      cp_async_wait_all();
      return -1;
    }
    if (lane < w) q.fd[j] = (unsigned short)(((tail + incl - k) << 4) | k);
    if (B >= head && B < head + w) {
      const int before = B - head;
      const int sb = __shfl_sync(0xffffffffu, incl, before > 0 ? before - 1 : 0);
      if (L >= kTileLv) {
        cp_async_wait_all();
        return -1;
      }
      ++L;
      B = tail + (before > 0 ? sb : 0);
      if (lane == 0) q.lev[L] = (unsigned short)B;
    }
    for (int e0 = 0; e0 < tot; e0 += 32) {
      const int e = e0 + lane;
      int s = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, s + step - 1);
        if (v <= e) s += step;
      }
      const int pm = __shfl_sync(0xffffffffu, msk, s);
      const int pc = __shfl_sync(0xffffffffu, c, s);
      const int pex = __shfl_sync(0xffffffffu, incl - k, s);
      if (e < tot) {
        const int kk = g_nth[pm * 8 + (e - pex)];
        const int pos = tail + e;
        const int cc = pc + off[kk];
        q.c[pos] = cc;
        q.pd[pos] = (1u << 16) | ((unsigned)(head + s) << 4) | (unsigned)(7 - kk);
        cp_async_elem(q.v + pos, lam + cc, true);
      }
    }
    tail += tot;
    head += w;
    __syncwarp();
  }
  // Alg 4: counts, deepest level first
  for (int l = L - 1; l >= 2; --l) {
    const int l0 = q.lev[l], l1 = q.lev[l + 1];
    for (int jj = l0 + lane; jj < l1; jj += 32) {
      const unsigned wd = q.pd[jj];
      atomicAdd(&q.pd[(wd >> 4) & 0xFFFu], wd & 0xFFFF0000u);
    }
    __syncwarp();
  }
  cp_async_wait_all();  // every entry's dL/dh' has arrived
  __syncwarp();
  // mu from the deepest level up: each entry adds its donors' mu * g in k
  // order, then writes its outputs
  for (int l = L - 1; l >= 0; --l) {
    const int l0 = q.lev[l], l1 = q.lev[l + 1];
    for (int jj = l0 + lane; jj < l1; jj += 32) {
      const unsigned f = q.fd[jj];
      const int d0 = (int)(f >> 4), nd = (int)(f & 15u);
      double mu = q.v[jj];
      if (nd) {
        // donors in k order; a donor's diagonal flag is its own code's
        double s = 0.0;
        for (int d = d0; d < d0 + nd; ++d) {
          const unsigned pdd = q.pd[d];
          double g, Gd;
          factors(a, (int)(pdd >> 16), nbr_diag((int)(pdd & 15u)), &g, &Gd);
          s += q.v[d] * g;
        }
        if (s != 0.0) mu += s;
        q.v[jj] = mu;
      }
      const unsigned pdj = q.pd[jj];
      cell_outputs(a, q.c[jj], (int)(pdj & 15u), (int)(pdj >> 16), mu);
    }
    __syncwarp();
  }
  return tail;
}

// The device-wide form of the step's sweep over all cells (queue, levels and
// counts of lem_levels/lem_accumulate order), one grid barrier per level.
__device__ bool adjoint_global(const AdjArgs& a, int L) {
  const StepArgs<double, int>& A = a.s;
  const unsigned G = gridDim.x;
  const int gtid = blockIdx.x * kBD + threadIdx.x, gstride = (int)G * kBD;
  for (int c = gtid; c < A.N; c += gstride) a.mu[c] = a.lam[c];
  if (!grid_barrier(A.st, G)) return false;
  for (int l = L - 2; l >= 0; --l) {
    const int lo = A.levels[l], hi = A.levels[l + 1];
    for (int j = lo + gtid; j < hi; j += gstride) {
      const int c = A.queue[j];
      int msk = A.mask[c];
      double s = 0.0;
      while (msk) {
        const int k = __ffs(msk) - 1;
        msk &= msk - 1;
        const int d = c + nbr_off(k, A.nx);
        double g, Gd;
        factors(a, A.cnt[d], nbr_diag(k), &g, &Gd);
        s += a.mu[d] * g;
      }
      if (s != 0.0) a.mu[c] += s;
    }
    if (!grid_barrier(A.st, G)) return false;
  }
  for (int c = gtid; c < A.N; c += gstride) cell_outputs(a, c, A.code[c], A.cnt[c], a.mu[c]);
  return true;
}

// One step of the sweep (see the file comment).
__global__ void __launch_bounds__(kBD, 1) adjoint_step_kernel(const __grid_constant__ AdjArgs a) {
  __shared__ Shared s;
  const StepArgs<double, int>& A = a.s;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const bool lead = blockIdx.x == 0 && t == 0;
  if (lead) A.st->dev_roots[0] = 0;  // overflow flag of this step (read after a barrier)
  if (!phase_codes(A)) return;
  if (ld_volatile(&A.st->err) != 0) return;  // a non-finite elevation: no outputs
  {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    const AdjTileQ q(dyn_smem + w * kWarpBytes);
    if (t < 8) s.off[t] = nbr_off(t, A.nx);
    fill_nth(t, kBD);
    __syncthreads();
    const int ntiles = A.tiles_x * ((A.ny + kAdjTileH - 1) / kAdjTileH);
    int tile = 0;
    if (lane == 0) tile = atomicAdd(&A.st->tiles_next[0], 1);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    while (tile < ntiles) {
      int next = 0;
      if (lane == 0) next = atomicAdd(&A.st->tiles_next[0], 1);
      const int r = tile_adjoint(a, q, s.off, tile, lane);
      if (r < 0 && lane == 0) atomicExch(&A.st->dev_roots[0], 1);
      tile = __shfl_sync(0xffffffffu, next, 0);
    }
  }
  if (!grid_barrier(A.st, gridDim.x)) return;
  if (lead) A.st->tiles_next[0] = 0;
  if (ld_volatile(&A.st->dev_roots[0]) != 0) {
    // some trees did not fit a warp: the whole step on device-wide levels
    if (lead) A.st->global_steps += 1;
    if (!phase_receivers(A, s)) return;
    const int L = phase_global_levels(A, s, A.levels[1], true);
    if (L < 0) return;
    if (!phase_global_accumulate(A, L)) return;
    if (!adjoint_global(a, L)) return;
    if (!grid_barrier(A.st, gridDim.x)) return;
  }
  // the step's terms into the running sums
  const int gtid = blockIdx.x * kBD + t, gstride = (int)gridDim.x * kBD;
  for (int c = gtid; c < A.N; c += gstride) {
    a.dLdU[c] += a.gU[c];
    a.dK_cell[c] += a.gK[c];
  }
}

// dL/dK = sum over cells of dK_cell, in a fixed order: block b sums its
// fixed range of cells with a fixed tree, the host the blocks in order.
constexpr int kSumBD = 256;
__global__ void __launch_bounds__(kSumBD) sum_cells_kernel(const double* v, int N, double* out) {
  __shared__ double red[kSumBD];
  const int per = (N + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * per, c1 = min(N, c0 + per);
  double acc = 0.0;
  for (int c = c0 + threadIdx.x; c < c1; c += kSumBD) acc += v[c];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kSumBD / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return LEM_OK;
  if (e == cudaErrorMemoryAllocation) return LEM_ENOMEM;
  return LEM_ECUDA;
}

#define ADJ_CUDA(call)            \
  do {                            \
    cudaError_t e_ = (call);      \
    if (e_ != cudaSuccess) {      \
      rc = status_of(e_);         \
      goto done;                  \
    }                             \
  } while (0)

#define ADJ_LEM(call)             \
  do {                            \
    rc = (call);                  \
    if (rc != LEM_OK) goto done;  \
  } while (0)

}  // namespace

// The step arguments of a context for the current binding (lem_api.cu).
int lem_make_step_args(lem_ctx* c, StepArgs<double, int>* a);

extern "C" LEM_API int lem_adjoint(lem_ctx* c, const double* dev_h0, const double* dev_lambda_T,
                                   int nsteps, int ckpt_every, double* dev_dLdU, double* dLdK,
                                   double* dev_lambda_0) {
  if (!c || !dev_h0 || !dev_lambda_T || !dev_dLdU || !dLdK || nsteps < 1 || ckpt_every < 1)
    return LEM_EINVAL;
  if (c->p.dtype != LEM_F64 || c->p.count_bits != 32) return LEM_EINVAL;
  if (c->newton_iters > 0) return LEM_EINVAL;  // the sweep below is the n-hat = 1 adjoint
  const size_t N = (size_t)c->N;
  const int nck = (nsteps + ckpt_every - 1) / ckpt_every;
  const int seglen = ckpt_every < nsteps ? ckpt_every : nsteps;
  constexpr int kSumBlocks = 256;
  int rc = LEM_OK;
  double *ck = nullptr, *seg = nullptr, *lam = nullptr, *lamp = nullptr, *mu = nullptr,
         *gU = nullptr, *gK = nullptr, *dKc = nullptr, *dks = nullptr;
  void* saved_h = c->h;
  std::vector<double> host_dk;
  ADJ_CUDA(cudaFuncSetAttribute((const void*)adjoint_step_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem));
  ADJ_CUDA(cudaMalloc(&ck, (size_t)nck * N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&seg, (size_t)(seglen + 1) * N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&lam, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&lamp, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&mu, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&gU, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&gK, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&dKc, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&dks, kSumBlocks * sizeof(double)));
  ADJ_CUDA(cudaMemsetAsync(dKc, 0, N * sizeof(double), c->stream));
  ADJ_CUDA(cudaMemsetAsync(dev_dLdU, 0, N * sizeof(double), c->stream));

  // forward pass from h0, keeping a checkpoint every ckpt_every steps
  ADJ_CUDA(cudaMemcpyAsync(seg, dev_h0, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  ADJ_LEM(lem_bind_elevation(c, seg, LEM_F64));
  for (int s = 0; s < nsteps; ++s) {
    if (s % ckpt_every == 0)
      ADJ_CUDA(cudaMemcpyAsync(ck + (size_t)(s / ckpt_every) * N, seg, N * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
    ADJ_LEM(lem_step(c, 1));
  }

  // reverse: each segment recomputed from its checkpoint, then swept back
  ADJ_CUDA(cudaMemcpyAsync(lam, dev_lambda_T, N * sizeof(double), cudaMemcpyDeviceToDevice,
                           c->stream));
  for (int k = nck - 1; k >= 0; --k) {
    const int s0 = k * ckpt_every;
    const int len = (s0 + ckpt_every < nsteps ? s0 + ckpt_every : nsteps) - s0;
    ADJ_CUDA(cudaMemcpyAsync(seg, ck + (size_t)k * N, N * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream));
    for (int i = 1; i <= len; ++i) {
      double* cur = seg + (size_t)i * N;
      ADJ_CUDA(cudaMemcpyAsync(cur, cur - N, N * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
      ADJ_LEM(lem_bind_elevation(c, cur, LEM_F64));
      ADJ_LEM(lem_step(c, 1));
    }
    for (int i = len; i >= 1; --i) {
      // step i maps seg[i-1] to seg[i]; its graph comes from seg[i-1]
      ADJ_LEM(lem_bind_elevation(c, seg + (size_t)(i - 1) * N, LEM_F64));
      AdjArgs a;
      ADJ_LEM(lem_make_step_args(c, &a.s));
      a.Gtab = c->Gtab;
      a.hnext = seg + (size_t)i * N;
      a.lam = lam;
      a.lam_prev = lamp;
      a.gU = gU;
      a.gK = gK;
      a.dLdU = dev_dLdU;
      a.dK_cell = dKc;
      a.mu = mu;
      void* args[] = {&a};
      ADJ_CUDA(cudaLaunchCooperativeKernel((const void*)adjoint_step_kernel, dim3(c->grid),
                                           dim3(kBD), args, kDynSmem, c->stream));
      double* tmp = lam;
      lam = lamp;
      lamp = tmp;
    }
  }
  ADJ_LEM(lem_sync(c));
  if (dev_lambda_0)
    ADJ_CUDA(cudaMemcpyAsync(dev_lambda_0, lam, N * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  sum_cells_kernel<<<kSumBlocks, kSumBD, 0, c->stream>>>(dKc, c->N, dks);
  ADJ_CUDA(cudaGetLastError());
  host_dk.resize(kSumBlocks);
  ADJ_CUDA(cudaMemcpyAsync(host_dk.data(), dks, kSumBlocks * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
  ADJ_CUDA(cudaStreamSynchronize(c->stream));
  {
    double sum = 0.0;
    for (int b = 0; b < kSumBlocks; ++b) sum += host_dk[b];
    *dLdK = sum;
  }
done:
  cudaStreamSynchronize(c->stream);
  // back to the caller's binding; stages derived from scratch states are stale
  if (saved_h) {
    const int rb = lem_bind_elevation(c, saved_h, c->p.dtype);
    if (rc == LEM_OK) rc = rb;
  } else {
    c->h = nullptr;
    c->tmap_ok = false;
  }
  if (!c->frozen) c->rec_valid = false;
  c->lev_valid = c->acc_valid = false;
  cudaFree(ck);
  cudaFree(seg);
  cudaFree(lam);
  cudaFree(lamp);
  cudaFree(mu);
  cudaFree(gU);
  cudaFree(gK);
  cudaFree(dKc);
  cudaFree(dks);
  return rc;
}
