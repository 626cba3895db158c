// lem_batch.cu -- many independent realizations of the landscape-evolution
// step (Barnes, arXiv:1803.02977) in one launch: the many-realization use the
// paper's abstract and closing sections motivate (inverse problems and
// statistics need many model runs; a GPU's spare capacity can run several
// models at once).
//
// Each thread block repeatedly claims the largest realization not yet taken
// (realizations are sorted by cell count; a device counter hands them out, so
// blocks are scheduled longest-first) and runs all of its time steps alone
// with block barriers: a realization's whole forest is the block's private
// forest, so no device-wide barrier is ever needed.  Elevations are FP32 with
// FP64 receiver slope tests (see receiver_code), erosion in the increment
// form with g = F/(1+F) from a per-realization shared-memory table.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "lem.h"
#include "lem_forest.cuh"

using namespace lem;

namespace {

constexpr int kBatchTN = 2048;  // counts tabulated per realization

struct BatchArgs {
  int R;
  const int* nx;
  const int* ny;
  const long long* off;    // cell offset of each realization (R+1)
  const double* Kdt;
  const double* m;
  const double* dx;
  const float* Udt;
  const int* order;        // realizations, largest first
  int* next;               // claim counter
  float* h;
  uint8_t* code;
  uint8_t* mask;
  int* pq;
  uint8_t* pqm;
  uint8_t* pqk;
  int* pqf;
  int* cntq;
  int* plev;               // level offsets: realization r at off[r] + r
  int nsteps;
};

template <int BD, int PI>
__global__ void __launch_bounds__(BD) lem_batch_kernel(BatchArgs a) {
  __shared__ ForestSmem<BD, PI> s;
  __shared__ float tab[2 * kBatchTN];
  __shared__ int s_r;
  const int t = threadIdx.x;
  while (true) {
    if (t == 0) {
      const int i = atomicAdd(a.next, 1);
      s_r = (i < a.R) ? a.order[i] : -1;
    }
    __syncthreads();
    const int r = s_r;
    __syncthreads();
    if (r < 0) break;
    const long long o = a.off[r];
    ForestGrid g;
    g.nx = a.nx[r];
    g.ny = a.ny[r];
    g.N = g.nx * g.ny;
    g.h = a.h + o;
    g.code = a.code + o;
    g.mask = a.mask + o;
    g.pq = a.pq + o;
    g.pqm = a.pqm + o;
    g.pqk = a.pqk + o;
    g.pqf = a.pqf + o;
    g.cntq = a.cntq + o;
    g.plev = a.plev + o + r;
    g.Udt = a.Udt[r];
    ErosionFactors ef;
    ef.tab = tab;
    ef.TN = kBatchTN;
    ef.Kdt = a.Kdt[r];
    ef.m = a.m[r];
    ef.dx = a.dx[r];
    ef.dxd = ef.dx * kSqrt2;
    ef.area = ef.dx * ef.dx;
    for (int i = t; i < kBatchTN; i += BD) {
      const double P = ef.Kdt * pow((double)i * ef.area, ef.m);
      const double Fc = P / ef.dx, Fd = P / ef.dxd;
      tab[i] = (float)(Fc / (1.0 + Fc));
      tab[kBatchTN + i] = (float)(Fd / (1.0 + Fd));
    }
    __syncthreads();
    for (int step = 0; step < a.nsteps; ++step) {
      const int n0 = forest_receivers<BD, PI>(g, s);
      const int PL = forest_levels<BD, PI>(g, n0, s);
      forest_accumulate<BD>(g, PL);
      forest_erode<BD>(g, PL, ef);
      __syncthreads();
    }
  }
}

struct Config {
  int bd, pi;
  const void* fn;
};

template <int BD, int PI>
Config config() {
  return Config{BD, PI, (const void*)&lem_batch_kernel<BD, PI>};
}

const Config kConfigs[] = {config<256, 4>(), config<256, 8>(), config<512, 4>(),
                           config<512, 8>(), config<1024, 4>(), config<1024, 8>()};

template <int BD, int PI>
cudaError_t launch(int grid, cudaStream_t s, BatchArgs& a) {
  lem_batch_kernel<BD, PI><<<grid, BD, 0, s>>>(a);
  return cudaGetLastError();
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return LEM_OK;
  if (e == cudaErrorMemoryAllocation) return LEM_ENOMEM;
  return LEM_ECUDA;
}

}  // namespace

struct lem_batch {
  int R = 0;
  long long total = 0;
  std::vector<long long> off;
  cudaStream_t stream = nullptr;
  int device = 0, nsm = 0;
  int cfg = 4;  // index into kConfigs
  int *d_nx = nullptr, *d_ny = nullptr, *d_order = nullptr, *d_next = nullptr;
  long long* d_off = nullptr;
  double *d_Kdt = nullptr, *d_m = nullptr, *d_dx = nullptr;
  float* d_Udt = nullptr;
  float* h = nullptr;
  uint8_t *code = nullptr, *mask = nullptr, *pqm = nullptr, *pqk = nullptr;
  int *pq = nullptr, *pqf = nullptr, *cntq = nullptr, *plev = nullptr;
};

extern "C" {

LEM_API void lem_batch_destroy(lem_batch* b) {
  if (!b) return;
  cudaFree(b->d_nx);
  cudaFree(b->d_ny);
  cudaFree(b->d_order);
  cudaFree(b->d_next);
  cudaFree(b->d_off);
  cudaFree(b->d_Kdt);
  cudaFree(b->d_m);
  cudaFree(b->d_dx);
  cudaFree(b->d_Udt);
  cudaFree(b->code);
  cudaFree(b->mask);
  cudaFree(b->pq);
  cudaFree(b->pqm);
  cudaFree(b->pqk);
  cudaFree(b->pqf);
  cudaFree(b->cntq);
  cudaFree(b->plev);
  delete b;
}

LEM_API int lem_batch_create(lem_batch** out, int R, const int* nx, const int* ny,
                             const double* dx, const double* K, const double* m,
                             const double* U, const double* dt, int dtype) {
  if (!out) return LEM_EINVAL;
  *out = nullptr;
  if (R < 1 || !nx || !ny || !dx || !K || !m || !U || !dt) return LEM_EINVAL;
  if (dtype != LEM_F32) return LEM_EINVAL;
  std::vector<long long> off(R + 1, 0);
  for (int r = 0; r < R; ++r) {
    if (nx[r] < 3 || ny[r] < 3) return LEM_EINVAL;
    if ((long long)nx[r] * ny[r] >= (1LL << 31) - 2) return LEM_EOVERFLOW;
    if (!(dx[r] > 0) || !(dt[r] > 0) || !(K[r] >= 0) || m[r] != m[r] || U[r] != U[r])
      return LEM_EINVAL;
    off[r + 1] = off[r] + (long long)nx[r] * ny[r];
  }
  lem_batch* b = new (std::nothrow) lem_batch();
  if (!b) return LEM_ENOMEM;
  b->R = R;
  b->off = off;
  b->total = off[R];
  std::vector<int> order(R);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) {
    return off[p + 1] - off[p] > off[q + 1] - off[q];
  });
  std::vector<double> Kdt(R), mm(R), ddx(R);
  std::vector<float> Udt(R);
  for (int r = 0; r < R; ++r) {
    Kdt[r] = K[r] * dt[r];
    mm[r] = m[r];
    ddx[r] = dx[r];
    Udt[r] = (float)(U[r] * dt[r]);
  }
  const size_t T = (size_t)b->total;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_nx, R * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ny, R * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_order, R * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_off, (R + 1) * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_Kdt, R * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_m, R * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_dx, R * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_Udt, R * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b->code, T);
  if (e == cudaSuccess) e = cudaMalloc(&b->mask, T);
  if (e == cudaSuccess) e = cudaMalloc(&b->pqm, T);
  if (e == cudaSuccess) e = cudaMalloc(&b->pqk, T);
  if (e == cudaSuccess) e = cudaMalloc(&b->pq, T * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->pqf, T * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->cntq, T * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->plev, (T + R) * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_nx, nx, R * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_ny, ny, R * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_order, order.data(), R * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_off, off.data(), (R + 1) * sizeof(long long), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_Kdt, Kdt.data(), R * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_m, mm.data(), R * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_dx, ddx.data(), R * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_Udt, Udt.data(), R * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    const int rc = status_of(e);
    lem_batch_destroy(b);
    return rc;
  }
  *out = b;
  return LEM_OK;
}

LEM_API int lem_batch_offsets(const lem_batch* b, int64_t* offsets) {
  if (!b || !offsets) return LEM_EINVAL;
  for (int r = 0; r <= b->R; ++r) offsets[r] = b->off[r];
  return LEM_OK;
}

LEM_API int lem_batch_set_stream(lem_batch* b, void* stream) {
  if (!b) return LEM_EINVAL;
  b->stream = (cudaStream_t)stream;
  return LEM_OK;
}

LEM_API int lem_batch_bind_elevation(lem_batch* b, float* dev_h) {
  if (!b || !dev_h) return LEM_EINVAL;
  b->h = dev_h;
  return LEM_OK;
}

LEM_API int lem_batch_set_config(lem_batch* b, int block_threads, int items_per_thread) {
  if (!b) return LEM_EINVAL;
  for (int i = 0; i < (int)(sizeof(kConfigs) / sizeof(kConfigs[0])); ++i) {
    if (kConfigs[i].bd == block_threads && kConfigs[i].pi == items_per_thread) {
      b->cfg = i;
      return LEM_OK;
    }
  }
  return LEM_EINVAL;
}

LEM_API int lem_batch_step(lem_batch* b, int nsteps) {
  if (!b || nsteps < 0) return LEM_EINVAL;
  if (!b->h) return LEM_ESTATE;
  if (nsteps == 0) return LEM_OK;
  const Config& c = kConfigs[b->cfg];
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c.fn, c.bd, 0);
  if (e != cudaSuccess) return status_of(e);
  if (per_sm < 1) return LEM_ECUDA;
  int grid = b->nsm * per_sm;
  if (grid > b->R) grid = b->R;
  e = cudaMemsetAsync(b->d_next, 0, sizeof(int), b->stream);
  if (e != cudaSuccess) return status_of(e);
  BatchArgs a;
  a.R = b->R;
  a.nx = b->d_nx;
  a.ny = b->d_ny;
  a.off = b->d_off;
  a.Kdt = b->d_Kdt;
  a.m = b->d_m;
  a.dx = b->d_dx;
  a.Udt = b->d_Udt;
  a.order = b->d_order;
  a.next = b->d_next;
  a.h = b->h;
  a.code = b->code;
  a.mask = b->mask;
  a.pq = b->pq;
  a.pqm = b->pqm;
  a.pqk = b->pqk;
  a.pqf = b->pqf;
  a.cntq = b->cntq;
  a.plev = b->plev;
  a.nsteps = nsteps;
  switch (b->cfg) {
    case 0: e = launch<256, 4>(grid, b->stream, a); break;
    case 1: e = launch<256, 8>(grid, b->stream, a); break;
    case 2: e = launch<512, 4>(grid, b->stream, a); break;
    case 3: e = launch<512, 8>(grid, b->stream, a); break;
    case 4: e = launch<1024, 4>(grid, b->stream, a); break;
    default: e = launch<1024, 8>(grid, b->stream, a); break;
  }
  return status_of(e);
}

LEM_API int lem_batch_sync(lem_batch* b) {
  if (!b) return LEM_EINVAL;
  return status_of(cudaStreamSynchronize(b->stream));
}

}  // extern "C"
