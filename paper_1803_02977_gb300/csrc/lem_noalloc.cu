// lem_noalloc.cu -- an allocation-free variant of the time-step entry point.
//
// Some callers cannot allocate device memory: a library embedded in a host
// framework whose caching allocator already owns the GPU's memory (an outside
// cudaMalloc would fail or fragment that pool), or a latency-critical loop in
// which cudaMalloc/cudaFree are not allowed because they can block and
// implicitly synchronise the device.  lem_step_noalloc serves them: the caller
// passes the elevations, and all the working memory of the step kernel (its
// receiver codes, donor masks, queues, counts, erosion tables and barrier
// words) lives in one file-scope __device__ array of fixed size, which every
// GPU that loads this library holds until the process exits.
//
// Host code cannot use the array's name as a device address (it names a host
// shadow), so the address is looked up once per device with
// cudaGetSymbolAddress, the first time the entry point is called on that
// device, with that device current.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "lem.h"
#include "lem_step_kernel.cuh"

using namespace lem;

namespace {

constexpr int kMaxCells = LEM_NOALLOC_MAX_CELLS;
constexpr int kMaxBlocks = 256;       // blocks of the cooperative grid used at most
// private-queue entries per block.  The context path sizes a block's share
// as max(2*ceil(N/grid), 4096); for N <= LEM_NOALLOC_MAX_CELLS and the
// 152-block grid of a GB300 that is 4096 as well (2*ceil(2^18/152) = 3450).
// On a GPU with fewer SMs the share is smaller than the context path's, which
// only sends more trees to the device-wide tier: the results are the same.
constexpr int kPcap = 4096;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Layout of the scratch array (each part 256-byte aligned).
constexpr size_t kOffState = 0;
constexpr size_t kOffPartial = kOffState + align256(sizeof(DevState));
constexpr size_t kOffFtab = kOffPartial + align256(sizeof(int) * kMaxBlocks);
constexpr size_t kOffGtab = kOffFtab + align256(sizeof(double2) * 2 * kTableN);
constexpr size_t kOffCode = kOffGtab + align256(sizeof(float) * 2 * kTableN);
constexpr size_t kOffMask = kOffCode + align256(kMaxCells + 2 * kCodeGuard);
constexpr size_t kOffQueue = kOffMask + align256(kMaxCells);
constexpr size_t kOffLevels = kOffQueue + align256(sizeof(int) * kMaxCells);
constexpr size_t kOffCnt = kOffLevels + align256(sizeof(int) * (kMaxCells + 2));
constexpr size_t kOffPq = kOffCnt + align256(sizeof(int) * kMaxCells);
constexpr size_t kOffPqm = kOffPq + align256(sizeof(int) * (size_t)kMaxBlocks * kPcap);
constexpr size_t kOffPqk = kOffPqm + align256((size_t)kMaxBlocks * kPcap);
constexpr size_t kOffPqf = kOffPqk + align256((size_t)kMaxBlocks * kPcap);
constexpr size_t kOffCntq = kOffPqf + align256(sizeof(int) * (size_t)kMaxBlocks * kPcap);
constexpr size_t kScratchBytes = kOffCntq + align256(sizeof(int) * (size_t)kMaxBlocks * kPcap);

// The shared working memory of every call on a device (about 20 MiB).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device, looked up on first use.
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Per-call set-up inside the scratch: clear the status and barrier words
// (they must start at zero) and fill the erosion tables for this call's
// parameters, with the same operation order as the step kernel expects.
__global__ void noalloc_prepare_kernel(unsigned char* base, int N, double Kdt, double m,
                                       double dx, double dxd, double area_scale) {
  DevState* st = reinterpret_cast<DevState*>(base + kOffState);
  // guard bytes around this call's receiver codes: never a valid code
  if (blockIdx.x == 0 && threadIdx.x < 2 * kCodeGuard) {
    const int i = threadIdx.x;
    base[kOffCode + (i < kCodeGuard ? i : kCodeGuard + N + (i - kCodeGuard))] = 0xFF;
  }
  double2* Ftab = reinterpret_cast<double2*>(base + kOffFtab);
  float* gtab = reinterpret_cast<float*>(base + kOffGtab);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    memset(st, 0, sizeof(DevState));
    st->wait_limit_ns = 2000000000ull;  // fixed 2 s bound on every device-side wait
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kTableN; i += gridDim.x * blockDim.x) {
    const double A = __dmul_rn((double)i, area_scale);
    const double P = __dmul_rn(Kdt, pow(A, m));
    const double Fc = __ddiv_rn(P, dx);
    const double Fd = __ddiv_rn(P, dxd);
    Ftab[i] = make_double2(Fc, __ddiv_rn(Fc, __dadd_rn(1.0, Fc)));
    Ftab[kTableN + i] = make_double2(Fd, __ddiv_rn(Fd, __dadd_rn(1.0, Fd)));
    gtab[i] = (float)(Fc / (1.0 + Fc));
    gtab[kTableN + i] = (float)(Fd / (1.0 + Fd));
  }
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return LEM_OK;
  if (e == cudaErrorMemoryAllocation) return LEM_ENOMEM;
  return LEM_ECUDA;
}

}  // namespace

extern "C" LEM_API int lem_step_noalloc(int nx, int ny, double* dev_h, double dx, double K,
                                        double m, double U, double dt, int nsteps,
                                        void* stream) {
  if (nx < 3 || ny < 3 || !dev_h || nsteps < 0) return LEM_EINVAL;
  if ((long long)nx * ny > kMaxCells) return LEM_EINVAL;  // beyond the fixed scratch
  if (!std::isfinite(dx) || !std::isfinite(K) || !std::isfinite(m) || !std::isfinite(U) ||
      !std::isfinite(dt) || dx <= 0 || dt <= 0 || K < 0)
    return LEM_EINVAL;
  if (nsteps == 0) return LEM_OK;
  cudaStream_t s = (cudaStream_t)stream;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  if (dev < 0 || dev >= kMaxDevices) return LEM_EINVAL;
  // the kernel runs on the current device: dev_h must be that device's memory
  // (a pointer to another GPU's memory would be dereferenced across devices)
  {
    cudaPointerAttributes pa;
    e = cudaPointerGetAttributes(&pa, dev_h);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return LEM_EINVAL;
    }
    if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
      return LEM_EINVAL;
  }
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return status_of(e);
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  unsigned char* base = g_scratch_addr[dev];

  int nsm = 0, per_sm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return status_of(e);
  e = cudaFuncSetAttribute((const void*)&lem_step_kernel<double, int>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
  if (e != cudaSuccess) return status_of(e);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, (const void*)&lem_step_kernel<double, int>, kBD, kDynSmem);
  if (e != cudaSuccess) return status_of(e);
  if (per_sm < 1) return LEM_ECUDA;
  int grid = nsm * per_sm;
  if (grid > kMaxBlocks) grid = kMaxBlocks;

  const double Kdt = K * dt, dxd = dx * kSqrt2, area = dx * dx;
  noalloc_prepare_kernel<<<64, 256, 0, s>>>(base, nx * ny, Kdt, m, dx, dxd, area);
  e = cudaGetLastError();
  if (e != cudaSuccess) return status_of(e);

  StepArgs<double, int> a;
  std::memset(&a, 0, sizeof(a));
  a.nx = nx;
  a.ny = ny;
  a.N = nx * ny;
  a.h = dev_h;
  a.Uf = nullptr;
  a.U = U;
  a.dt = dt;
  a.Kdt = Kdt;
  a.m = m;
  a.dx = dx;
  a.dxd = dxd;
  a.area_scale = area;
  a.code = base + kOffCode + kCodeGuard;
  a.mask = base + kOffMask;
  a.queue = reinterpret_cast<int*>(base + kOffQueue);
  a.levels = reinterpret_cast<int*>(base + kOffLevels);
  a.pq = reinterpret_cast<int*>(base + kOffPq);
  a.pqm = base + kOffPqm;
  a.pqk = base + kOffPqk;
  a.pqf = reinterpret_cast<int*>(base + kOffPqf);
  a.cntq = reinterpret_cast<int*>(base + kOffCntq);
  a.pcap = kPcap;
  a.Udt = U * dt;
  a.Udt_f = (float)(U * dt);
  a.cnt = reinterpret_cast<int*>(base + kOffCnt);
  a.Ftab = reinterpret_cast<const double2*>(base + kOffFtab);
  a.gtab = reinterpret_cast<const float*>(base + kOffGtab);
  a.st = reinterpret_cast<DevState*>(base + kOffState);
  a.partial = reinterpret_cast<int*>(base + kOffPartial);
  a.tiles_x = (nx + kTileW - 1) / kTileW;
  a.ntiles = a.tiles_x * ((ny + tile_h<double>() - 1) / tile_h<double>());
  a.strip_rows = pick_strip_rows<double>(nx, ny, grid * kWarps);
  a.has_tmap = 0;  // strips are staged with per-element asynchronous copies
  a.phases = kPhTiles;
  a.nsteps = nsteps;
  a.frozen = 0;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)&lem_step_kernel<double, int>, dim3(grid),
                                  dim3(kBD), args, kDynSmem, s);
  if (e != cudaSuccess) return status_of(e);

  // wait for the step and report the kernel's own status word
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return status_of(e);
  int err = 0;
  e = cudaMemcpy(&err, base + kOffState + offsetof(DevState, err), sizeof(int),
                 cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return status_of(e);
  return err;
}
