// lem_api.cu -- the C ABI declared in include/lem.h: context management,
// argument and state checks, cooperative launches of the persistent step
// kernel, and the small kernels that convert the internal compact arrays to
// the paper's exported layouts (Table 1: Rec, Donor/Dnum, Queue, Levels,
// Accum).
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)

#include "lem.h"
#include "lem_context.cuh"
#include "lem_step_kernel.cuh"

using namespace lem;

int lem_fill_launch(lem_ctx* c);



namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LEM_OK;
  if (e == cudaErrorMemoryAllocation) return LEM_ENOMEM;
  return LEM_ECUDA;
}

#define LEM_CUDA(call)                        \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

// Erosion factors by cell count: F = K*dt*(count*area_scale)^m / d with the
// same operation order as the per-cell expression, g = F/(1+F) by FP64
// division, g rounded once to float, and dF/dK = dt*A^m/d for the adjoint.
__global__ void build_tables_kernel(double2* Ftab, float* gtab, double2* Gtab, double Kdt,
                                    double dt, double m, double dx, double dxd,
                                    double area_scale) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kTableN; i += gridDim.x * blockDim.x) {
    const double A = __dmul_rn((double)i, area_scale);
    const double Am = pow(A, m);
    const double Gp = __dmul_rn(dt, Am);
    Gtab[i] = make_double2(__ddiv_rn(Gp, dx), __ddiv_rn(Gp, dxd));
    const double P = __dmul_rn(Kdt, Am);
    const double Fc = __ddiv_rn(P, dx);
    const double Fd = __ddiv_rn(P, dxd);
    Ftab[i] = make_double2(Fc, __ddiv_rn(Fc, __dadd_rn(1.0, Fc)));
    Ftab[kTableN + i] = make_double2(Fd, __ddiv_rn(Fd, __dadd_rn(1.0, Fd)));
    gtab[i] = (float)(Fc / (1.0 + Fc));
    gtab[kTableN + i] = (float)(Fd / (1.0 + Fd));
  }
}

__global__ void export_rec_kernel(const uint8_t* __restrict__ code, int32_t* __restrict__ rec,
                                  int N, int nx) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const int k = code[c];
    rec[c] = no_receiver(k) ? c : c + nbr_off(k, nx);
  }
}

__global__ void export_donors_kernel(const uint8_t* __restrict__ mask, int32_t* __restrict__ dnum,
                                     int32_t* __restrict__ donor, int N, int nx) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    int msk = mask[c];
    if (dnum) dnum[c] = __popc(msk);
    if (donor) {
      int i = 0;
      while (msk) {
        const int k = __ffs(msk) - 1;
        msk &= msk - 1;
        donor[8LL * c + i++] = c + nbr_off(k, nx);
      }
      for (; i < 8; ++i) donor[8LL * c + i] = -1;
    }
  }
}

__global__ void export_levels_kernel(const int* __restrict__ levels, int64_t* __restrict__ out,
                                     int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = levels[i];
}

__global__ void export_depth_kernel(const int* __restrict__ queue, const int* __restrict__ levels,
                                    int L, int32_t* __restrict__ depth, int N) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    int lo = 0, hi = L;  // find l with levels[l] <= j < levels[l+1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (levels[mid] <= j) lo = mid; else hi = mid;
    }
    depth[queue[j]] = lo;
  }
}

// Frozen receivers: int32 addresses -> codes; invalid entries are an error.
__global__ void import_rec_kernel(const int32_t* __restrict__ rec, uint8_t* __restrict__ code,
                                  int N, int nx, int ny, DevState* st) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
    const int r = rec[c];
    const int x = c % nx, y = c / nx;
    const bool perim = (x == 0 || y == 0 || x == nx - 1 || y == ny - 1);
    int k = perim ? kEdge : kSink;
    if (r != c) {
      if (perim || r < 0 || r >= N) {
        set_error(st, kErrInval);
      } else {
        const int ddx = r % nx - x, ddy = r / nx - y;
        for (int q = 0; q < 8; ++q)
          if (nbr_dx(q) == ddx && nbr_dy(q) == ddy) k = q;
        if (k >= kSink) set_error(st, kErrInval);
      }
    }
    code[c] = (uint8_t)k;
  }
}

// Waits on a flag nothing sets, bounded by the context's wait limit.
__global__ void selftest_wait_kernel(DevState* st) {
  if (threadIdx.x != 0) return;
  const unsigned long long t0 = global_ns();
  while (ld_volatile(&st->selftest_flag) == 0) {
    if (global_ns() - t0 > st->wait_limit_ns) {
      set_error(st, kErrTimeout);
      return;
    }
  }
}

template <typename HT, typename CT>
const void* step_kernel_ptr(bool newton) {
  return newton ? (const void*)&lem_step_kernel<HT, CT, true>
                : (const void*)&lem_step_kernel<HT, CT, false>;
}

// The step kernel of a context's element and count types; newton: the
// instantiation for a general slope exponent.
const void* kernel_for(const lem_ctx* c, bool newton) {
  const bool f64 = c->p.dtype == LEM_F64, c64 = c->p.count_bits == 64;
  if (f64) return c64 ? step_kernel_ptr<double, long long>(newton)
                      : step_kernel_ptr<double, int>(newton);
  return c64 ? step_kernel_ptr<float, long long>(newton) : step_kernel_ptr<float, int>(newton);
}

// Rows per strip of the codes pass: the lem_set_tiling choice, else the
// heuristic (pick_strip_rows).
int strip_rows_of(const lem_ctx* c) {
  if (c->strip_rows > 0) return c->strip_rows;
  return c->p.dtype == LEM_F64 ? pick_strip_rows<double>(c->p.nx, c->p.ny, c->grid * kWarps)
                               : pick_strip_rows<float>(c->p.nx, c->p.ny, c->grid * kWarps);
}

template <typename HT, typename CT>
StepArgs<HT, CT> make_args(lem_ctx* c, int phases, int nsteps) {
  StepArgs<HT, CT> a;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.N = c->N;
  a.h = (HT*)c->h;
  a.Uf = c->Uf;
  a.U = c->p.U;
  a.dt = c->p.dt;
  a.Kdt = c->Kdt;
  a.m = c->p.m;
  a.dx = c->p.dx;
  a.dxd = c->dxd;
  a.area_scale = c->area_scale;
  a.code = c->code;
  a.mask = c->mask;
  a.queue = c->queue;
  a.levels = c->levels;
  a.cnt = (CT*)c->cnt;
  a.Ftab = c->Ftab;
  a.gtab = c->gtab;
  a.st = c->st;
  a.partial = c->partial;
  a.pq = c->pq;
  a.pqm = c->pqm;
  a.pqk = c->pqk;
  a.pqf = c->pqf;
  a.cntq = (CT*)c->cntq;
  a.pcap = c->pcap;
  a.tiles_x = (c->p.nx + kTileW - 1) / kTileW;
  a.ntiles = a.tiles_x * ((c->p.ny + tile_h<HT>() - 1) / tile_h<HT>());
  a.strip_rows = strip_rows_of(c);
  a.half_tiles = c->half_tiles;
  a.has_tmap = c->tmap_ok ? 1 : 0;
  a.tmap = c->tmap;
  a.Udt = c->p.U * c->p.dt;
  a.Udt_f = (float)(c->p.U * c->p.dt);
  a.phases = phases;
  a.nsteps = nsteps;
  a.frozen = c->frozen ? 1 : 0;
  a.newton_iters = c->newton_iters;
  a.nexp = c->nexp;
  a.neps = c->neps;
  a.dxn = c->dxn;
  a.dxdn = c->dxdn;
  a.dfac = c->dfac;
  a.dfacd = c->dfacd;
  a.jt = c->jt;
  a.jab1 = c->jab1;
  a.jp0 = c->jp0;
  a.jp1 = c->jp1;
  a.jstamp = c->jstamp;
  // breadth-first levels before jumping: a device-wide level costs several
  // microseconds, a jumping round over the whole grid grows with its size
  a.jump_cap = c->N >> 15 > 64 ? c->N >> 15 : 64;
  // with the jumping tier, forests deeper than 256 levels leave the block
  // tier for it (a block-private level costs about a microsecond and more)
  a.priv_levels = c->jt ? 256 : kMaxPrivLevels;
  return a;
}

// Scratch of the pointer-jumping device tier (lem_jump.cuh), allocated once:
// tour words, a second (A, B) buffer, two pointer buffers, root stamps.
int ensure_jump_scratch(lem_ctx* c) {
  if (c->jt) return LEM_OK;
  const size_t N = (size_t)c->N;
  unsigned long long* jt = nullptr;
  double2* ab = nullptr;
  int *p0 = nullptr, *p1 = nullptr;
  unsigned* stamp = nullptr;
  cudaError_t e = cudaMalloc(&jt, 2 * N * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&ab, N * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&p0, N * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&p1, N * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&stamp, N * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(stamp, 0, N * sizeof(unsigned), c->stream);
  if (e != cudaSuccess) {
    cudaFree(jt);
    cudaFree(ab);
    cudaFree(p0);
    cudaFree(p1);
    cudaFree(stamp);
    return cuda_status(e);
  }
  c->jt = jt;
  c->jab1 = ab;
  c->jp0 = p0;
  c->jp1 = p1;
  c->jstamp = stamp;
  return LEM_OK;
}

template <typename HT, typename CT>
int launch_typed(lem_ctx* c, int phases, int nsteps) {
  StepArgs<HT, CT> a = make_args<HT, CT>(c, phases, nsteps);
  void* args[] = {&a};
  LEM_CUDA(cudaLaunchCooperativeKernel(step_kernel_ptr<HT, CT>(c->newton_iters > 0), dim3(c->grid),
                                       dim3(kBD), args, kDynSmem, c->stream));
  return LEM_OK;
}

int launch_step(lem_ctx* c, int phases, int nsteps) {
  const bool f64 = c->p.dtype == LEM_F64, c64 = c->p.count_bits == 64;
  if (f64) return c64 ? launch_typed<double, long long>(c, phases, nsteps)
                      : launch_typed<double, int>(c, phases, nsteps);
  return c64 ? launch_typed<float, long long>(c, phases, nsteps)
             : launch_typed<float, int>(c, phases, nsteps);
}

int aux_grid(const lem_ctx* c) {
  long long blocks = ((long long)c->N + 255) / 256;
  return (int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
}

// Read the sticky status (and L) back; synchronises the stream.
int read_status(lem_ctx* c, int* nlevels) {
  LEM_CUDA(cudaMemcpyAsync(c->host_status, &c->st->err, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  const int err = c->host_status[0];
  if (nlevels) *nlevels = c->host_status[1];
  if (err != 0) {
    // an abandoned barrier may have left arrivals counted: start clean
    LEM_CUDA(cudaMemsetAsync(&c->st->bar_count, 0, sizeof(unsigned), c->stream));
    LEM_CUDA(cudaMemsetAsync(&c->st->err, 0, sizeof(int), c->stream));
    LEM_CUDA(cudaMemsetAsync(c->st->tiles_next, 0, sizeof(c->st->tiles_next), c->stream));
    LEM_CUDA(cudaStreamSynchronize(c->stream));
    return err;
  }
  return LEM_OK;
}

bool is_finite(double v) { return std::isfinite(v); }

// Encode the TMA descriptor of the bound elevations (2-D: nx x ny elements,
// box kStageCols x (strip rows + 4), zero fill outside) into c->tmap; every launch
// passes it in its kernel parameter.  Leaves c->tmap_ok false -- the step kernel then
// stages strips with per-element copies -- when TMA cannot describe h (row
// pitch or base not a multiple of 16 bytes) or the driver lacks the encoder.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_tmap(lem_ctx* c) {
  c->tmap_ok = false;
  if (!c->h) return LEM_OK;
  const size_t esz = c->p.dtype == LEM_F64 ? 8 : 4;
  const size_t pitch = (size_t)c->p.nx * esz;
  if (pitch % 16 != 0 || ((uintptr_t)c->h) % 16 != 0) return LEM_OK;
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return LEM_OK;
    }
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[2] = {(cuuint64_t)c->p.nx, (cuuint64_t)c->p.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch};
  const int rows = strip_rows_of(c) + 4;
  const cuuint32_t box[2] = {(cuuint32_t)kStageCols, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(&m, esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                            2, c->h, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return LEM_OK;
  static_assert(sizeof(m) == sizeof(c->tmap), "descriptor size");
  std::memcpy(&c->tmap, &m, sizeof(m));
  c->tmap_ok = true;
  return LEM_OK;
}

}  // namespace

// The step arguments of a context for its current binding, for the other
// translation units' launches (the adjoint sweep).
int lem_make_step_args(lem_ctx* c, StepArgs<double, int>* a) {
  if (!c || !a || c->p.dtype != LEM_F64 || c->p.count_bits != 32) return LEM_EINVAL;
  *a = make_args<double, int>(c, 0, 1);
  return LEM_OK;
}

extern "C" {

const char* lem_status_string(int s) {
  switch (s) {
    case LEM_OK: return "ok";
    case LEM_EINVAL: return "invalid argument, receiver graph or non-finite elevation";
    case LEM_ENOMEM: return "device allocation failed";
    case LEM_ECUDA: return "CUDA runtime error";
    case LEM_ETIMEOUT: return "bounded device wait ran out";
    case LEM_ESTATE: return "stage called before its inputs were computed";
    case LEM_EOVERFLOW: return "grid too large for 32-bit cell addresses";
    case LEM_EBOUNDS: return "index out of bounds (checked build)";
    default: return "unknown status";
  }
}

int lem_create(lem_ctx** out, int nx, int ny, double dx, double K, double m, double U,
               double dt) {
  lem_params p;
  std::memset(&p, 0, sizeof(p));
  p.nx = nx;
  p.ny = ny;
  p.dx = dx;
  p.K = K;
  p.m = m;
  p.U = U;
  p.dt = dt;
  p.area_scale = 0.0;
  p.dtype = LEM_F64;
  p.count_bits = 32;
  return lem_create_ex(out, &p);
}

int lem_create_ex(lem_ctx** out, const lem_params* pin) {
  if (!out) return LEM_EINVAL;
  *out = nullptr;
  if (!pin) return LEM_EINVAL;
  const lem_params p = *pin;
  if (p.nx < 3 || p.ny < 3) return LEM_EINVAL;
  if ((long long)p.nx * p.ny >= (1LL << 31) - 2) return LEM_EOVERFLOW;
  if (!is_finite(p.dx) || p.dx <= 0 || !is_finite(p.dt) || p.dt <= 0 || !is_finite(p.K) || p.K < 0 ||
      !is_finite(p.m) || !is_finite(p.U) || !is_finite(p.area_scale))
    return LEM_EINVAL;
  if (p.dtype != LEM_F64 && p.dtype != LEM_F32) return LEM_EINVAL;
  if (p.count_bits != 32 && p.count_bits != 64) return LEM_EINVAL;

  lem_ctx* c = new (std::nothrow) lem_ctx();
  if (!c) return LEM_ENOMEM;
  c->p = p;
  c->N = p.nx * p.ny;
  c->Kdt = p.K * p.dt;
  c->dxd = p.dx * kSqrt2;
  c->area_scale = p.area_scale > 0 ? p.area_scale : p.dx * p.dx;
  int rc = LEM_OK;
  cudaError_t e = cudaGetDevice(&c->device);
  const size_t N = (size_t)c->N;
  int nsm = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
  for (int nw = 0; nw < 2 && e == cudaSuccess; ++nw)
    e = cudaFuncSetAttribute(kernel_for(c, nw != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kDynSmem);
  // both instantiations are launched with this grid: it must suit either
  int per_sm_newton = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(c, false), kBD,
                                                      kDynSmem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_newton, kernel_for(c, true), kBD,
                                                      kDynSmem);
  if (e == cudaSuccess && per_sm_newton < per_sm) per_sm = per_sm_newton;
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) {
    c->grid = nsm * (per_sm < 2 ? per_sm : 2);
    // private queue share: twice the fair share of cells, at least 4096
    const long long fair = ((long long)c->N + c->grid - 1) / c->grid;
    c->pcap = (int)(2 * fair > 4096 ? 2 * fair : 4096);
    // receiver codes with kCodeGuard bytes of 0xFF on both sides (never a
    // valid code): word loads of neighbouring rows stay in bounds
    e = cudaMalloc(&c->code_base, N + 2 * kCodeGuard);
    if (e == cudaSuccess) e = cudaMemset(c->code_base, 0xFF, N + 2 * kCodeGuard);
    c->code = c->code_base + kCodeGuard;
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->mask, N);
  if (e == cudaSuccess) e = cudaMalloc(&c->queue, N * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->levels, (N + 2) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->cnt, N * (p.count_bits / 8));
  if (e == cudaSuccess) e = cudaMalloc(&c->Ftab, 2 * kTableN * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&c->gtab, 2 * kTableN * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&c->Gtab, kTableN * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&c->st, sizeof(DevState));
  if (e == cudaSuccess) e = cudaMalloc(&c->partial, (size_t)c->grid * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->pq, (size_t)c->grid * c->pcap * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->pqm, (size_t)c->grid * c->pcap);
  if (e == cudaSuccess) e = cudaMalloc(&c->pqk, (size_t)c->grid * c->pcap);
  if (e == cudaSuccess) e = cudaMalloc(&c->pqf, (size_t)c->grid * c->pcap * sizeof(int));
  if (e == cudaSuccess)
    e = cudaMalloc(&c->cntq, (size_t)c->grid * c->pcap * (p.count_bits / 8));
  if (e == cudaSuccess) e = cudaMallocHost(&c->host_status, 4 * sizeof(int));
  if (e == cudaSuccess) {
    DevState s;
    std::memset(&s, 0, sizeof(s));
    s.wait_limit_ns = (unsigned long long)(c->wait_limit_s * 1e9);
    e = cudaMemcpy(c->st, &s, sizeof(s), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    build_tables_kernel<<<64, 256>>>(c->Ftab, c->gtab, c->Gtab, c->Kdt, p.dt, p.m, p.dx, c->dxd,
                                     c->area_scale);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    rc = cuda_status(e);
    lem_destroy(c);
    return rc;
  }
  *out = c;
  return LEM_OK;
}

void lem_destroy(lem_ctx* c) {
  if (!c) return;
  cudaFree(c->code_base);
  cudaFree(c->mask);
  cudaFree(c->queue);
  cudaFree(c->levels);
  cudaFree(c->cnt);
  cudaFree(c->Ftab);
  cudaFree(c->gtab);
  cudaFree(c->Gtab);
  cudaFree(c->st);
  cudaFree(c->partial);
  cudaFree(c->pq);
  cudaFree(c->pqm);
  cudaFree(c->pqk);
  cudaFree(c->pqf);
  cudaFree(c->cntq);
  cudaFree(c->trace);
  cudaFree(c->fill_w);
  cudaFree(c->fill_dirty);
  cudaFree(c->fill_state);
  cudaFree(c->fill_ptr);
  cudaFree(c->mfd_pending);
  cudaFree(c->mfd_norm);
  cudaFree(c->mfd_queue);
  cudaFree(c->mfd_state);
  cudaFree(c->jt);
  cudaFree(c->jab1);
  cudaFree(c->jp0);
  cudaFree(c->jp1);
  cudaFree(c->jstamp);
  if (c->host_status) cudaFreeHost(c->host_status);
  delete c;
}

int lem_set_stream(lem_ctx* c, void* stream) {
  if (!c) return LEM_EINVAL;
  c->stream = (cudaStream_t)stream;
  return LEM_OK;
}

int lem_bind_elevation(lem_ctx* c, void* dev_h, int dtype) {
  if (!c || !dev_h || dtype != c->p.dtype) return LEM_EINVAL;
  c->h = dev_h;
  const int rc = encode_tmap(c);
  if (rc != LEM_OK) return rc;
  if (!c->frozen) c->rec_valid = false;
  c->lev_valid = c->frozen && c->lev_valid;
  c->acc_valid = c->frozen && c->acc_valid;
  return LEM_OK;
}

int lem_set_uplift_field(lem_ctx* c, const double* dev_U) {
  if (!c) return LEM_EINVAL;
  c->Uf = dev_U;
  return LEM_OK;
}

int lem_receivers(lem_ctx* c, int32_t* dev_rec) {
  if (!c) return LEM_EINVAL;
  if (!c->h && !c->frozen) return LEM_ESTATE;
  int rc = launch_step(c, kPhRec, 1);
  if (rc != LEM_OK) return rc;
  c->rec_valid = true;
  c->graph_valid = true;
  c->lev_valid = c->acc_valid = false;
  if (dev_rec) {
    export_rec_kernel<<<aux_grid(c), 256, 0, c->stream>>>(c->code, dev_rec, c->N, c->p.nx);
    LEM_CUDA(cudaGetLastError());
  }
  return LEM_OK;
}

int lem_donors(lem_ctx* c, int32_t* dev_dnum, int32_t* dev_donor) {
  if (!c) return LEM_EINVAL;
  if (!c->rec_valid) return LEM_ESTATE;
  if (dev_dnum || dev_donor) {
    export_donors_kernel<<<aux_grid(c), 256, 0, c->stream>>>(c->mask, dev_dnum, dev_donor, c->N,
                                                             c->p.nx);
    LEM_CUDA(cudaGetLastError());
  }
  return LEM_OK;
}

int lem_levels(lem_ctx* c, int64_t* nlevels, int32_t* dev_queue, int64_t* dev_levels,
               int32_t* dev_depth) {
  if (!c) return LEM_EINVAL;
  if (!c->rec_valid) return LEM_ESTATE;
  int rc = launch_step(c, kPhLev, 1);
  if (rc != LEM_OK) return rc;
  int L = 0;
  rc = read_status(c, &L);
  if (rc != LEM_OK) {
    c->lev_valid = false;
    return rc;
  }
  c->lev_valid = true;
  c->acc_valid = false;
  if (nlevels) *nlevels = L;
  if (dev_queue)
    LEM_CUDA(cudaMemcpyAsync(dev_queue, c->queue, (size_t)c->N * sizeof(int),
                             cudaMemcpyDeviceToDevice, c->stream));
  if (dev_levels) {
    export_levels_kernel<<<1 + L / 256, 256, 0, c->stream>>>(c->levels, dev_levels, L + 1);
    LEM_CUDA(cudaGetLastError());
  }
  if (dev_depth) {
    export_depth_kernel<<<aux_grid(c), 256, 0, c->stream>>>(c->queue, c->levels, L, dev_depth,
                                                            c->N);
    LEM_CUDA(cudaGetLastError());
  }
  return LEM_OK;
}

int lem_accumulate(lem_ctx* c, void* dev_counts) {
  if (!c) return LEM_EINVAL;
  if (!c->lev_valid) return LEM_ESTATE;
  int rc = launch_step(c, kPhAcc, 1);
  if (rc != LEM_OK) return rc;
  c->acc_valid = true;
  if (dev_counts)
    LEM_CUDA(cudaMemcpyAsync(dev_counts, c->cnt, (size_t)c->N * (c->p.count_bits / 8),
                             cudaMemcpyDeviceToDevice, c->stream));
  return LEM_OK;
}

int lem_erode(lem_ctx* c) {
  if (!c) return LEM_EINVAL;
  if (!c->h) return LEM_ESTATE;
  if (!c->acc_valid) return LEM_ESTATE;
  int rc = launch_step(c, kPhEro, 1);
  if (rc != LEM_OK) return rc;
  if (!c->frozen) c->rec_valid = c->lev_valid = c->acc_valid = false;
  return LEM_OK;
}

int lem_step(lem_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return LEM_EINVAL;
  if (!c->h) return LEM_ESTATE;
  if (nsteps == 0) return LEM_OK;
  if (c->mode == 0 && c->newton_iters == 0 && c->N < (1 << 30)) {
    const int rj = ensure_jump_scratch(c);
    if (rj != LEM_OK) return rj;
  }
  if (c->fill_on) {
    // one step at a time: the depression flood, then the step
    for (int s = 0; s < nsteps; ++s) {
      int rc = lem_fill_launch(c);
      if (rc == LEM_OK) rc = launch_step(c, c->mode == 0 ? kPhTiles : kPhAll, 1);
      if (rc != LEM_OK) return rc;
    }
    c->graph_valid = true;
    c->rec_valid = c->frozen;
    c->lev_valid = c->acc_valid = c->frozen && c->mode == 1;
    return LEM_OK;
  }
  int rc = launch_step(c, c->mode == 0 ? kPhTiles : kPhAll, nsteps);
  if (rc != LEM_OK) return rc;
  c->graph_valid = true;
  // A frozen graph's codes and masks stay current; the device-wide queue and
  // counts are current only if the device-wide form ran (mode 1).
  c->rec_valid = c->frozen;
  c->lev_valid = c->acc_valid = c->frozen && c->mode == 1;
  return LEM_OK;
}

int lem_set_slope_exponent(lem_ctx* c, double n, double eps, int max_iter) {
  if (!c || !is_finite(n) || n < 1.0) return LEM_EINVAL;
  if (n == 1.0) {
    c->newton_iters = 0;
    c->nexp = 1.0;
    c->neps = c->dxn = c->dxdn = c->dfac = c->dfacd = 0.0;
    return LEM_OK;
  }
  if (!is_finite(eps) || !(eps > 0.0) || max_iter < 1 || max_iter > 1000) return LEM_EINVAL;
  c->newton_iters = max_iter;
  c->nexp = n;
  c->neps = eps;
  c->dxn = std::pow(c->p.dx, n);
  c->dxdn = std::pow(c->dxd, n);
  c->dfac = std::pow(c->p.dx, 1.0 - n);
  c->dfacd = std::pow(c->dxd, 1.0 - n);
  return LEM_OK;
}

int lem_set_receivers(lem_ctx* c, const int32_t* dev_rec) {
  if (!c) return LEM_EINVAL;
  c->rec_valid = c->lev_valid = c->acc_valid = false;
  if (!dev_rec) {
    c->frozen = false;
    return LEM_OK;
  }
  import_rec_kernel<<<aux_grid(c), 256, 0, c->stream>>>(dev_rec, c->code, c->N, c->p.nx, c->p.ny,
                                                        c->st);
  LEM_CUDA(cudaGetLastError());
  int rc = read_status(c, nullptr);
  if (rc != LEM_OK) {
    c->frozen = false;
    return rc;
  }
  c->frozen = true;
  rc = launch_step(c, kPhRec, 1);  // donor masks and level 0 of the frozen graph
  if (rc != LEM_OK) return rc;
  c->rec_valid = true;
  return LEM_OK;
}

int lem_last_graph(lem_ctx* c, int32_t* dev_rec, uint8_t* dev_mask) {
  if (!c) return LEM_EINVAL;
  if (!c->graph_valid) return LEM_ESTATE;
  if (dev_rec) {
    export_rec_kernel<<<aux_grid(c), 256, 0, c->stream>>>(c->code, dev_rec, c->N, c->p.nx);
    LEM_CUDA(cudaGetLastError());
  }
  if (dev_mask)
    LEM_CUDA(cudaMemcpyAsync(dev_mask, c->mask, (size_t)c->N, cudaMemcpyDeviceToDevice,
                             c->stream));
  return LEM_OK;
}

// ---- checkpoint / resume --------------------------------------------------
// A state blob: a header (format tag, grid, element type, steps taken, the
// device tier's jumping hint) followed by the bound elevations.
namespace {
struct StateHeader {
  uint32_t tag;        // 'LEMS'
  uint32_t version;    // 1
  int32_t nx, ny;
  int32_t dtype;       // LEM_F64 or LEM_F32
  int32_t jump_hint;   // the device tier starts with pointer jumping
  int64_t steps;       // lem_step steps taken by the context (private + device-wide)
};
static_assert(sizeof(StateHeader) == 32, "state header layout");
constexpr uint32_t kStateTag = 0x534D454Cu;  // "LEMS" in memory order

size_t state_bytes(const lem_ctx* c) {
  return sizeof(StateHeader) + (size_t)c->N * (c->p.dtype == LEM_F64 ? 8 : 4);
}
}  // namespace

int lem_state_size(lem_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return LEM_EINVAL;
  *bytes = (int64_t)state_bytes(c);
  return LEM_OK;
}

int lem_get_state(lem_ctx* c, void* buf, int64_t bytes) {
  if (!c || !buf) return LEM_EINVAL;
  if (!c->h) return LEM_ESTATE;
  if (bytes < (int64_t)state_bytes(c)) return LEM_EINVAL;
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  int w[2] = {0, 0};
  LEM_CUDA(cudaMemcpy(&w[0], (char*)c->st + offsetof(DevState, private_steps), sizeof(int),
                      cudaMemcpyDeviceToHost));
  LEM_CUDA(cudaMemcpy(&w[1], (char*)c->st + offsetof(DevState, global_steps), sizeof(int),
                      cudaMemcpyDeviceToHost));
  int hint = 0;
  LEM_CUDA(cudaMemcpy(&hint, (char*)c->st + offsetof(DevState, jump_hint), sizeof(int),
                      cudaMemcpyDeviceToHost));
  StateHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  hd.tag = kStateTag;
  hd.version = 1;
  hd.nx = c->p.nx;
  hd.ny = c->p.ny;
  hd.dtype = c->p.dtype;
  hd.jump_hint = hint;
  hd.steps = (int64_t)w[0] + w[1];
  LEM_CUDA(cudaMemcpy(buf, &hd, sizeof(hd), cudaMemcpyDefault));
  LEM_CUDA(cudaMemcpy((char*)buf + sizeof(hd), c->h, state_bytes(c) - sizeof(hd),
                      cudaMemcpyDefault));
  return LEM_OK;
}

int lem_set_state(lem_ctx* c, const void* buf, int64_t bytes) {
  if (!c || !buf) return LEM_EINVAL;
  if (!c->h) return LEM_ESTATE;
  if (bytes < (int64_t)state_bytes(c)) return LEM_EINVAL;
  StateHeader hd;
  LEM_CUDA(cudaMemcpy(&hd, buf, sizeof(hd), cudaMemcpyDefault));
  if (hd.tag != kStateTag || hd.version != 1 || hd.nx != c->p.nx || hd.ny != c->p.ny ||
      hd.dtype != c->p.dtype || hd.steps < 0 || (hd.jump_hint != 0 && hd.jump_hint != 1))
    return LEM_EINVAL;
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  LEM_CUDA(cudaMemcpy(c->h, (const char*)buf + sizeof(hd), state_bytes(c) - sizeof(hd),
                      cudaMemcpyDefault));
  // the step counter resumes as private steps (the split is not kept)
  const int w[2] = {(int)hd.steps, 0};
  LEM_CUDA(cudaMemcpy((char*)c->st + offsetof(DevState, private_steps), &w[0], sizeof(int),
                      cudaMemcpyHostToDevice));
  LEM_CUDA(cudaMemcpy((char*)c->st + offsetof(DevState, global_steps), &w[1], sizeof(int),
                      cudaMemcpyHostToDevice));
  LEM_CUDA(cudaMemcpy((char*)c->st + offsetof(DevState, jump_hint), &hd.jump_hint, sizeof(int),
                      cudaMemcpyHostToDevice));
  if (!c->frozen) c->rec_valid = false;
  c->lev_valid = c->acc_valid = false;
  return LEM_OK;
}

int lem_sync(lem_ctx* c) {
  if (!c) return LEM_EINVAL;
  return read_status(c, nullptr);
}

int lem_set_wait_limit(lem_ctx* c, double seconds) {
  if (!c || !(seconds > 0) || !is_finite(seconds)) return LEM_EINVAL;
  c->wait_limit_s = seconds;
  unsigned long long ns = (unsigned long long)(seconds * 1e9);
  LEM_CUDA(cudaMemcpyAsync(&c->st->wait_limit_ns, &ns, sizeof(ns), cudaMemcpyHostToDevice,
                           c->stream));
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  return LEM_OK;
}

int lem_set_step_mode(lem_ctx* c, int mode) {
  if (!c || (mode != 0 && mode != 1)) return LEM_EINVAL;
  c->mode = mode;
  return LEM_OK;
}

int lem_set_tiling(lem_ctx* c, int rows, int half_tiles) {
  if (!c || (half_tiles != 0 && half_tiles != 1)) return LEM_EINVAL;
  const int most = c->p.dtype == LEM_F64 ? lem::strip_rows<double>() : lem::strip_rows<float>();
  if (rows != 0 && rows != 8 && rows != 16 && rows != 32) return LEM_EINVAL;
  if (rows > most) return LEM_EINVAL;
  c->strip_rows = rows;
  c->half_tiles = half_tiles;
  return encode_tmap(c);  // the strips' TMA box follows the rows
}

int lem_get_tiling(lem_ctx* c, int* rows, int* half_tiles) {
  if (!c || !rows || !half_tiles) return LEM_EINVAL;
  *rows = strip_rows_of(c);
  *half_tiles = c->half_tiles;
  return LEM_OK;
}

int lem_step_stats(lem_ctx* c, int64_t* private_steps, int64_t* device_wide_steps) {
  if (!c) return LEM_EINVAL;
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  int v[2] = {0, 0};
  LEM_CUDA(cudaMemcpy(&v[0], (char*)c->st + offsetof(DevState, private_steps), sizeof(int),
                      cudaMemcpyDeviceToHost));
  LEM_CUDA(cudaMemcpy(&v[1], (char*)c->st + offsetof(DevState, global_steps), sizeof(int),
                      cudaMemcpyDeviceToHost));
  if (private_steps) *private_steps = v[0];
  if (device_wide_steps) *device_wide_steps = v[1];
  return LEM_OK;
}

int lem_jump_stats(lem_ctx* c, int64_t* stats) {
  if (!c || !stats) return LEM_EINVAL;
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  int v[2] = {0, 0};
  LEM_CUDA(cudaMemcpy(&v[0], (char*)c->st + offsetof(DevState, jump_steps), sizeof(int),
                      cudaMemcpyDeviceToHost));
  LEM_CUDA(cudaMemcpy(&v[1], (char*)c->st + offsetof(DevState, jump_rounds), sizeof(int),
                      cudaMemcpyDeviceToHost));
  stats[0] = v[0];
  stats[1] = v[1];
  return LEM_OK;
}

int lem_tier_stats(lem_ctx* c, int64_t* cells) {
  if (!c || !cells) return LEM_EINVAL;
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  unsigned long long v[3] = {0, 0, 0};
  LEM_CUDA(cudaMemcpy(v, (char*)c->st + offsetof(DevState, tier_cells), sizeof(v),
                      cudaMemcpyDeviceToHost));
  for (int i = 0; i < 3; ++i) cells[i] = (int64_t)v[i];
  return LEM_OK;
}

int lem_trace_enable(lem_ctx* c, int capacity) {
  if (!c || capacity < 0) return LEM_EINVAL;
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  if (c->trace) {
    cudaFree(c->trace);
    c->trace = nullptr;
  }
  if (capacity > 0) LEM_CUDA(cudaMalloc(&c->trace, 2 * sizeof(unsigned long long) * capacity));
  const int capn[2] = {capacity, 0};  // trace_cap, trace_n (adjacent)
  LEM_CUDA(cudaMemcpy((char*)c->st + offsetof(DevState, trace), &c->trace, sizeof(c->trace),
                      cudaMemcpyHostToDevice));
  LEM_CUDA(cudaMemcpy((char*)c->st + offsetof(DevState, trace_cap), capn, sizeof(capn),
                      cudaMemcpyHostToDevice));
  return LEM_OK;
}

int lem_trace_read(lem_ctx* c, int64_t* ns, int32_t* tags, int cap, int* n) {
  if (!c || cap < 0 || (cap > 0 && (!ns || !tags))) return LEM_EINVAL;
  LEM_CUDA(cudaStreamSynchronize(c->stream));
  int cnt = 0, tcap = 0;
  LEM_CUDA(cudaMemcpy(&tcap, (char*)c->st + offsetof(DevState, trace_cap), sizeof(int),
                      cudaMemcpyDeviceToHost));
  LEM_CUDA(cudaMemcpy(&cnt, (char*)c->st + offsetof(DevState, trace_n), sizeof(int),
                      cudaMemcpyDeviceToHost));
  if (n) *n = cnt;
  int m = cnt < cap ? cnt : cap;
  if (m > tcap) m = tcap;
  if (m > 0) {
    std::vector<unsigned long long> buf(2 * (size_t)m);
    LEM_CUDA(cudaMemcpy(buf.data(), c->trace, buf.size() * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost));
    for (int i = 0; i < m; ++i) {
      ns[i] = (int64_t)buf[2 * i];
      tags[i] = (int32_t)buf[2 * i + 1];
    }
  }
  const int zero = 0;
  LEM_CUDA(cudaMemcpy((char*)c->st + offsetof(DevState, trace_n), &zero, sizeof(int),
                      cudaMemcpyHostToDevice));
  return LEM_OK;
}

int lem_selftest_wait(lem_ctx* c) {
  if (!c) return LEM_EINVAL;
  selftest_wait_kernel<<<1, 32, 0, c->stream>>>(c->st);
  LEM_CUDA(cudaGetLastError());
  return read_status(c, nullptr);
}

}  // extern "C"
