// lem_batch.cu -- many independent realizations of the landscape-evolution
// step (Barnes, arXiv:1803.02977) in one launch: the many-realization use the
// paper's abstract and closing sections motivate (inverse problems and
// statistics need many model runs; a GPU's spare capacity can run several
// models at once).
//
// Each thread block repeatedly claims the largest realization not yet taken
// (realizations are sorted by cell count; a device counter hands them out, so
// blocks are scheduled longest-first) and runs all of its time steps alone
// with block barriers, so no device-wide barrier is ever needed.  Inside a
// realization the step takes the same tiered form as lem_step: the block's
// warps compute receiver codes and donor masks strip by strip (Algs 1-2),
// then run Algs 3-6 on warp-private tile forests in shared memory; tiles
// whose forest does not fit are finished on the block-wide forest of the
// realization (lem_forest.cuh), whose queue holds the whole grid.
// Elevations are FP32 with FP64 receiver slope tests for near ties, erosion
// in the increment form with g = F/(1+F) from a per-realization table.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "lem.h"
#include "lem_forest.cuh"
#include "lem_tiles.cuh"

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
  const float* gtab;       // F/(1+F) by count: realization r at r * 2 * kBatchTN
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

// g = F/(1+F) for counts below kBatchTN, F = K*dt*(count*dx^2)^m / d (the
// same operation order as the single-grid tables).
__global__ void batch_tables_kernel(float* gtab, int R, const double* Kdt, const double* m,
                                    const double* dx) {
  const long long total = (long long)R * kBatchTN;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / kBatchTN), cnt = (int)(i - (long long)r * kBatchTN);
    const double ddx = dx[r], ddd = ddx * kSqrt2, area = ddx * ddx;
    const double P = Kdt[r] * pow((double)cnt * area, m[r]);
    const double Fc = P / ddx, Fd = P / ddd;
    gtab[(size_t)r * 2 * kBatchTN + cnt] = (float)(Fc / (1.0 + Fc));
    gtab[(size_t)r * 2 * kBatchTN + kBatchTN + cnt] = (float)(Fd / (1.0 + Fd));
  }
}

template <int BD, int PI>
__global__ void __launch_bounds__(BD) lem_batch_kernel(BatchArgs a) {
  constexpr int TH = tile_h<float>();
  __shared__ ForestSmem<BD, PI> s;
  __shared__ int s_r, s_next, s_n_ovf, s_n0;
  __shared__ int s_off[8];
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  float* S = reinterpret_cast<float*>(dyn_smem + w * kWarpBytes);
  const TileQ<float> q(dyn_smem + w * kWarpBytes);
  fill_nth(t, BD);  // read after the block barrier below
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
    // the warp slices are idle while the block forest runs
    g.splev = reinterpret_cast<int*>(dyn_smem);
    g.splev_cap = (BD / 32) * kWarpBytes / (int)sizeof(int);
    g.Udt = a.Udt[r];
    const float* tab = a.gtab + (size_t)r * 2 * kBatchTN;
    ErosionFactors ef;
    ef.tab = tab;
    ef.TN = kBatchTN;
    ef.Kdt = a.Kdt[r];
    ef.m = a.m[r];
    ef.dx = a.dx[r];
    ef.dxd = ef.dx * kSqrt2;
    ef.area = ef.dx * ef.dx;
    TileArgs<float> ta;
    ta.nx = g.nx;
    ta.ny = g.ny;
    ta.tiles_x = (g.nx + kTileW - 1) / kTileW;
    ta.code = g.code;
    ta.mask = g.mask;
    ta.h = g.h;
    ta.ero.gtab = tab;
    ta.ero.tn = kBatchTN;
    ta.ero.Uf = nullptr;
    ta.ero.Udt = (double)g.Udt;
    ta.ero.dt = 0.0;
    ta.ero.Udt_f = g.Udt;
    const int ntiles = ta.tiles_x * ((g.ny + TH - 1) / TH);
    const int nsx = (g.nx + kStripOut - 1) / kStripOut;
    const int rows = pick_strip_rows<float>(g.nx, g.ny, BD / 32);
    const int units = nsx * ((g.ny + rows - 1) / rows);
    if (t < 8) s_off[t] = nbr_off(t, g.nx);
    for (int step = 0; step < a.nsteps; ++step) {
      // Algs 1-2: the realization's strips, claimed by the block's warps
      if (t == 0) s_next = 0;
      __syncthreads();
      while (true) {
        int u = 0;
        if (lane == 0) u = atomicAdd(&s_next, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= units) break;
        const int sy = u / nsx, sx = u - sy * nsx;
        const int x0 = sx * kStripOut, y0 = sy * rows;
        const int xb = (x0 - 2) & ~3;
        stage_strip(g.h, g.nx, g.ny, xb, y0 - 2, rows + 4, S, lane);
        codes_strip(S, g.code, g.mask, g.nx, g.ny, x0, y0, rows, xb, false, lane);
        __syncwarp();
      }
      __syncthreads();
      // Algs 3-6 on warp-private tile forests; tiles that do not fit are
      // listed in pqf (free until the block-wide forest runs)
      if (t == 0) {
        s_next = 0;
        s_n_ovf = 0;
        s_n0 = 0;
      }
      __syncthreads();
      while (true) {
        int tile = 0;
        if (lane == 0) tile = atomicAdd(&s_next, 1);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (tile >= ntiles) break;
        if (tile_forest(ta, q, s_off, tile_item(tile, 0), lane) < 0 && lane == 0)
          g.pqf[atomicAdd(&s_n_ovf, 1)] = tile;
      }
      __syncthreads();
      const int nov = s_n_ovf;
      if (nov > 0) {
        // their roots as level 0 of the block-wide forest
        for (int i = w; i < nov; i += BD / 32) {
          int cd[TH], x, y0;
          tile_codes<TH>(g.code, g.pqf[i], 0, TH, ta.tiles_x, g.nx, g.ny, lane, cd, &x, &y0);
#pragma unroll
          for (int rr = 0; rr < TH; ++rr) {
            const bool f = cd[rr] >= kSink;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (bal == 0) continue;
            int base = 0;
            if (lane == 0) base = atomicAdd(&s_n0, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (f) {
              const int pos = base + __popc(bal & ((1u << lane) - 1u));
              const int c = (y0 + rr) * g.nx + x;
              g.pq[pos] = c;
              g.pqm[pos] = g.mask[c];
              g.pqk[pos] = (uint8_t)cd[rr];
            }
          }
        }
        __syncthreads();
        const int PL = forest_levels<BD, PI>(g, s_n0, s);
        forest_accumulate<BD>(g, PL);
        forest_erode<BD>(g, PL, ef);
      }
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

// dynamic shared memory of a block: one warp slice per warp
constexpr int dyn_smem_of(int bd) { return (bd / 32) * kWarpBytes; }

template <int BD, int PI>
cudaError_t launch(int grid, cudaStream_t s, BatchArgs& a) {
  lem_batch_kernel<BD, PI><<<grid, BD, dyn_smem_of(BD), s>>>(a);
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
  float* gtab = nullptr;  // erosion factors per realization (batch_tables_kernel)
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
  cudaFree(b->gtab);
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
  if (e == cudaSuccess) e = cudaMalloc(&b->gtab, (size_t)R * 2 * kBatchTN * sizeof(float));
  if (e == cudaSuccess) {
    batch_tables_kernel<<<256, 256>>>(b->gtab, R, b->d_Kdt, b->d_m, b->d_dx);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
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
  cudaError_t e = cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       dyn_smem_of(c.bd));
  if (e != cudaSuccess) return status_of(e);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c.fn, c.bd, dyn_smem_of(c.bd));
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
  a.gtab = b->gtab;
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
