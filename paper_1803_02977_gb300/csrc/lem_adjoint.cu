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
// The sweep uses the device-wide breadth-first levels (lem_levels), one grid
// barrier per level, pulling each cell's donors from the level above.
#include <cmath>
#include <cstring>
#include <vector>

#include "lem.h"
#include "lem_context.cuh"

using namespace lem;

namespace {

struct AdjArgs {
  int nx, N, L;
  const uint8_t* code;
  const uint8_t* mask;
  const int* queue;
  const int* levels;
  const int* cnt;
  const double2* Ftab;  // {F, g} by count
  const double2* Gtab;  // {dF/dK cardinal, dF/dK diagonal} by count
  double Kdt, m, dx, dxd, area_scale, dt;
  const double* hnext;
  const double* lam;
  double* mu;
  double* lam_prev;
  double* dLdU;
  double* dK_partial;  // one per block, accumulated across steps
  DevState* st;
};

constexpr int kABD = 512;

__device__ __forceinline__ void factors(const AdjArgs& a, int count, bool diag, double* g,
                                        double* G) {
  if (count < kTableN) {
    *g = a.Ftab[(diag ? kTableN : 0) + count].y;
    const double2 gg = a.Gtab[count];
    *G = diag ? gg.y : gg.x;
    return;
  }
  const double Am = pow((double)count * a.area_scale, a.m);
  const double d = diag ? a.dxd : a.dx;
  const double F = a.Kdt * Am / d;
  *g = F / (1.0 + F);
  *G = a.dt * Am / d;
}

__global__ void __launch_bounds__(kABD) adjoint_step_kernel(AdjArgs a) {
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, t = threadIdx.x;
  const int gtid = b * kABD + t, gstride = (int)G * kABD;
  __shared__ double s_red[kABD / 32];
  for (int c = gtid; c < a.N; c += gstride) a.mu[c] = a.lam[c];
  if (!grid_barrier(a.st, G)) return;
  // donors first: level L-2 down to 0 pulls from the level above
  for (int l = a.L - 2; l >= 0; --l) {
    const int lo = a.levels[l], hi = a.levels[l + 1];
    for (int j = lo + gtid; j < hi; j += gstride) {
      const int c = a.queue[j];
      int msk = a.mask[c];
      double s = 0.0;
      while (msk) {
        const int k = __ffs(msk) - 1;
        msk &= msk - 1;
        const int d = c + nbr_off(k, a.nx);
        double g, Gd;
        factors(a, a.cnt[d], nbr_diag(k), &g, &Gd);
        s += a.mu[d] * g;
      }
      if (s != 0.0) a.mu[c] += s;
    }
    if (!grid_barrier(a.st, G)) return;
  }
  double dk = 0.0;
  for (int c = gtid; c < a.N; c += gstride) {
    const int k = a.code[c];
    const double mu = a.mu[c];
    if (k == kEdge) {
      a.lam_prev[c] = mu;
    } else if (k == kSink) {
      a.lam_prev[c] = mu;
      a.dLdU[c] += a.dt * mu;
    } else {
      double g, Gc;
      factors(a, a.cnt[c], nbr_diag(k), &g, &Gc);
      const double w = mu * (1.0 - g);  // mu / (1 + F)
      a.lam_prev[c] = w;
      a.dLdU[c] += a.dt * w;
      dk += w * (a.hnext[c + nbr_off(k, a.nx)] - a.hnext[c]) * Gc;
    }
  }
  // block sum in a fixed order, added to this block's running partial
  const int lane = t & 31, w = t >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dk += __shfl_down_sync(0xffffffffu, dk, o);
  if (lane == 0) s_red[w] = dk;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int i = 0; i < kABD / 32; ++i) s += s_red[i];
    a.dK_partial[b] += s;
  }
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

extern "C" LEM_API int lem_adjoint(lem_ctx* c, const double* dev_h0, const double* dev_lambda_T,
                                   int nsteps, int ckpt_every, double* dev_dLdU, double* dLdK,
                                   double* dev_lambda_0) {
  if (!c || !dev_h0 || !dev_lambda_T || !dev_dLdU || !dLdK || nsteps < 1 || ckpt_every < 1)
    return LEM_EINVAL;
  if (c->p.dtype != LEM_F64 || c->p.count_bits != 32) return LEM_EINVAL;
  const size_t N = (size_t)c->N;
  const int nck = (nsteps + ckpt_every - 1) / ckpt_every;
  const int seglen = ckpt_every < nsteps ? ckpt_every : nsteps;
  int per_sm = 0, nsm = 0, grid = 0, rc = LEM_OK;
  double *ck = nullptr, *seg = nullptr, *lam = nullptr, *lamp = nullptr, *mu = nullptr,
         *dkp = nullptr;
  void* saved_h = c->h;
  std::vector<double> host_dk;
  ADJ_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  ADJ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_step_kernel, kABD, 0));
  if (per_sm < 1) {
    rc = LEM_ECUDA;
    goto done;
  }
  grid = nsm * (per_sm < 2 ? per_sm : 2);
  ADJ_CUDA(cudaMalloc(&ck, (size_t)nck * N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&seg, (size_t)(seglen + 1) * N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&lam, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&lamp, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&mu, N * sizeof(double)));
  ADJ_CUDA(cudaMalloc(&dkp, (size_t)grid * sizeof(double)));
  ADJ_CUDA(cudaMemsetAsync(dkp, 0, (size_t)grid * sizeof(double), c->stream));
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
      // the graph of step i, from its input elevations
      ADJ_LEM(lem_bind_elevation(c, seg + (size_t)(i - 1) * N, LEM_F64));
      ADJ_LEM(lem_receivers(c, nullptr));
      int64_t L = 0;
      ADJ_LEM(lem_levels(c, &L, nullptr, nullptr, nullptr));
      ADJ_LEM(lem_accumulate(c, nullptr));
      AdjArgs a;
      a.nx = c->p.nx;
      a.N = c->N;
      a.L = (int)L;
      a.code = c->code;
      a.mask = c->mask;
      a.queue = c->queue;
      a.levels = c->levels;
      a.cnt = (const int*)c->cnt;
      a.Ftab = c->Ftab;
      a.Gtab = c->Gtab;
      a.Kdt = c->Kdt;
      a.m = c->p.m;
      a.dx = c->p.dx;
      a.dxd = c->dxd;
      a.area_scale = c->area_scale;
      a.dt = c->p.dt;
      a.hnext = seg + (size_t)i * N;
      a.lam = lam;
      a.mu = mu;
      a.lam_prev = lamp;
      a.dLdU = dev_dLdU;
      a.dK_partial = dkp;
      a.st = c->st;
      void* args[] = {&a};
      ADJ_CUDA(cudaLaunchCooperativeKernel((const void*)adjoint_step_kernel, dim3(grid),
                                           dim3(kABD), args, 0, c->stream));
      double* tmp = lam;
      lam = lamp;
      lamp = tmp;
    }
  }
  ADJ_LEM(lem_sync(c));
  if (dev_lambda_0)
    ADJ_CUDA(cudaMemcpyAsync(dev_lambda_0, lam, N * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream));
  host_dk.resize(grid);
  ADJ_CUDA(cudaMemcpyAsync(host_dk.data(), dkp, (size_t)grid * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
  ADJ_CUDA(cudaStreamSynchronize(c->stream));
  {
    double s = 0.0;
    for (int b = 0; b < grid; ++b) s += host_dk[b];
    *dLdK = s;
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
  cudaFree(dkp);
  return rc;
}
