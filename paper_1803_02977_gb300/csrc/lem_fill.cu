// lem_fill.cu -- depression filling before Alg 1 (Section "Local Minima":
// depressions filled to the level of their outlets, the flats this leaves
// resolved as part of the flood, as Priority-Flood with epsilon increments
// does).  The filled surface w is the least one with w >= h, w = h on the
// perimeter and every interior cell strictly above its lowest neighbour:
//     w[c] = max(h[c], next value above min over the 8 neighbours of w).
// That fixed point is unique, and relaxing w[c] <- max(h[c], next(min)) from
// w = +inf in the interior decreases monotonically onto it in any order, so
// the order of the parallel relaxation does not change a single bit of the
// result.
//
// One cooperative launch.  The grid is cut into 32 x 32 tiles; in each round
// warps claim tiles from a device-wide counter, and a warp relaxes a dirty
// tile alone: it stages w (with a one-cell halo, the neighbours' latest
// values read from L2) and h in its slice of shared memory, sweeps the tile
// down, up, right and left until a pass changes nothing, writes the changed
// tile back and marks its eight neighbour tiles dirty for the next round.
// Rounds end at a bounded grid barrier; the flood is done after a round in
// which no tile changed.
//
// The start need not be +inf everywhere: any w0 >= T(w0) (T the right-hand
// side above) decreases onto the same fixed point.  w0 = h is such a start at
// every cell whose chain of lowest strictly lower neighbours ends on the
// perimeter (each cell of the chain has a neighbour below it that keeps its
// h), so the kernel first finds every chain's end by pointer jumping and
// starts from +inf only in the basins of interior pits and flats.  Only the
// tiles holding such cells are relaxed in the first round.
//
// The relaxation runs on order-preserving integer keys of the elevations
// (FillKey): min and max become integer operations and the next value up is
// key + 1, which equals IEEE nextafter(x, +inf) for every finite x (-0 is
// taken as +0).  GB300 runs FP64 arithmetic at a small fraction of its
// integer rate, and the flood needs no arithmetic beyond these orderings.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>

#include "lem.h"
#include "lem_context.cuh"

namespace lem {

constexpr int kFT = 32;        // tile edge (one lane per column or row)
constexpr int kFS = kFT + 2;   // staged edge: the tile and its halo
constexpr int kFillPasses = 64;  // relaxation passes per tile visit, at most

// warps per block: the staged w and h of every warp fill ~209 KB of shared
// memory with either element type
template <typename HT>
__host__ __device__ constexpr int fill_warps() {
  return sizeof(HT) == 8 ? 12 : 24;
}
template <typename HT>
__host__ __device__ constexpr int fill_warp_bytes() {
  return (kFS * kFS + kFT * kFT) * (int)sizeof(HT);
}

// Order-preserving keys: for non-NaN x, key(x) < key(y) iff x < y (with -0
// mapped to +0); the largest key is +inf's.
template <typename HT> struct FillKey;
template <> struct FillKey<double> {
  using K = unsigned long long;
  static constexpr K kSign = 0x8000000000000000ull;
  static constexpr K kInf = 0xFFF0000000000000ull;  // key of +inf
  __device__ static K of(double x) {
    K b = (K)__double_as_longlong(x);
    if (b == kSign) b = 0;  // -0 as +0
    return (b & kSign) ? ~b : (b | kSign);
  }
  __device__ static double value(K k) {
    return __longlong_as_double((long long)((k & kSign) ? (k ^ kSign) : ~k));
  }
};
template <> struct FillKey<float> {
  using K = unsigned int;
  static constexpr K kSign = 0x80000000u;
  static constexpr K kInf = 0xFF800000u;
  __device__ static K of(float x) {
    K b = __float_as_uint(x);
    if (b == kSign) b = 0;
    return (b & kSign) ? ~b : (b | kSign);
  }
  __device__ static float value(K k) { return __uint_as_float((k & kSign) ? (k ^ kSign) : ~k); }
};

// Round bookkeeping, triple-buffered by round so that a word is reset two
// barriers after its last use.
struct FillState {
  int claim[3];  // tiles claimed in the round
  int mark[3];   // some tile was marked dirty for the next round
  int jump[3];   // some pointer moved in the pointer-jumping pass
  int rounds;    // rounds the last flood took
  int visits;    // tile visits (dirty tiles relaxed) in the last flood
  unsigned long long passes;  // relaxation passes over all visits
  int unsettled;  // visits that ran out of passes
};

template <typename HT>
struct FillArgs {
  int nx, ny, tiles_x, ntiles, max_rounds;
  HT* h;           // in: the surface; out: the filled surface
  typename FillKey<HT>::K* w;  // scratch: keys of the relaxed surface, nx*ny
  int* ptr;        // scratch: lowest lower neighbour, then the chain's end
  uint8_t* dirty;  // two arrays of ntiles flags, by round parity (zero on entry)
  FillState* fs;
  DevState* st;
};

template <typename K>
__device__ __forceinline__ K kmin(K a, K b) {
  return a < b ? a : b;
}

// One relaxation of tile cell (ly, lx) in key space: returns true if w went
// down.  Every lane reads its nine staged keys before any lane writes (the
// __syncwarp between), so lanes never race on shared memory.
template <typename K>
__device__ __forceinline__ bool relax_cell(K* sW, const K* sH, int ly, int lx, int gx, int gy,
                                           int nx, int ny, K kinf) {
  K* p = sW + (ly + 1) * kFS + (lx + 1);
  const bool interior = gx > 0 && gx < nx - 1 && gy > 0 && gy < ny - 1;
  K v = p[0];
  if (interior) {
    const K lo = kmin(kmin(kmin(p[-kFS - 1], p[-kFS]), kmin(p[-kFS + 1], p[-1])),
                      kmin(kmin(p[1], p[kFS - 1]), kmin(p[kFS], p[kFS + 1])));
    const K up = lo == kinf ? lo : lo + 1;  // the next value above lo
    const K hk = sH[ly * kFT + lx];
    v = hk > up ? hk : up;
  }
  const bool down = v < p[0];
  __syncwarp();
  if (down) p[0] = v;
  __syncwarp();
  return down;
}

// Relax one tile with one warp until a pass changes nothing (or
// kFillPasses).  Returns 1 if the tile changed, 2 if it also did not settle.
template <typename HT>
__device__ int fill_tile(const FillArgs<HT>& a, int tile, typename FillKey<HT>::K* sW,
                         typename FillKey<HT>::K* sH, int lane) {
  using FK = FillKey<HT>;
  using K = typename FK::K;
  const int nx = a.nx, ny = a.ny;
  const int ty = tile / a.tiles_x, tx = tile - ty * a.tiles_x;
  const int x0 = tx * kFT, y0 = ty * kFT;
  for (int i = lane; i < kFS * kFS; i += 32) {
    const int r = i / kFS, col = i - r * kFS;
    const int gx = x0 - 1 + col, gy = y0 - 1 + r;
    sW[i] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny) ? __ldcg(a.w + (size_t)gy * nx + gx)
                                                       : FK::kInf;
  }
  for (int i = lane; i < kFT * kFT; i += 32) {
    const int r = i / kFT, col = i - r * kFT;
    const int gx = x0 + col, gy = y0 + r;
    sH[i] = (gx < nx && gy < ny) ? FK::of(a.h[(size_t)gy * nx + gx]) : K(0);
  }
  __syncwarp();
  bool changed = false;
  int pass = 0;
  for (; pass < kFillPasses; ++pass) {
    bool ch = false;
    // lane = column: down the tile, then up
    for (int y = 0; y < kFT; ++y)
      ch |= relax_cell<K>(sW, sH, y, lane, x0 + lane, y0 + y, nx, ny, FK::kInf);
    for (int y = kFT - 1; y >= 0; --y)
      ch |= relax_cell<K>(sW, sH, y, lane, x0 + lane, y0 + y, nx, ny, FK::kInf);
    // lane = row: rightward, then leftward
    for (int x = 0; x < kFT; ++x)
      ch |= relax_cell<K>(sW, sH, lane, x, x0 + x, y0 + lane, nx, ny, FK::kInf);
    for (int x = kFT - 1; x >= 0; --x)
      ch |= relax_cell<K>(sW, sH, lane, x, x0 + x, y0 + lane, nx, ny, FK::kInf);
    if (!__any_sync(0xffffffffu, ch)) break;
    changed = true;
  }
  if (changed) {
    for (int i = lane; i < kFT * kFT; i += 32) {
      const int r = i / kFT, col = i - r * kFT;
      const int gx = x0 + col, gy = y0 + r;
      if (gx < nx && gy < ny) __stcg(a.w + (size_t)gy * nx + gx, sW[(r + 1) * kFS + col + 1]);
    }
  }
  if (lane == 0) {
    atomicAdd(&a.fs->visits, 1);
    atomicAdd(&a.fs->passes, (unsigned long long)(pass + (pass < kFillPasses ? 1 : 0)));
    if (pass == kFillPasses) atomicAdd(&a.fs->unsettled, 1);
  }
  return changed ? (pass == kFillPasses ? 2 : 1) : 0;
}

template <typename HT>
__global__ void __launch_bounds__(fill_warps<HT>() * 32, 1)
    fill_kernel(const __grid_constant__ FillArgs<HT> a) {
  extern __shared__ __align__(16) unsigned char fill_smem[];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  using FK = FillKey<HT>;
  using K = typename FK::K;
  K* sW = reinterpret_cast<K*>(fill_smem + wi * fill_warp_bytes<HT>());
  K* sH = sW + kFS * kFS;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  const int nx = a.nx, ny = a.ny;
  const long long N = (long long)nx * ny;
  const unsigned G = gridDim.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gstride = (long long)G * blockDim.x;
  // each cell's lowest strictly lower neighbour (lowest k among equals), or
  // itself: perimeter cells, and interior pits and flats
  for (long long c = gtid; c < N; c += gstride) {
    const int y = (int)(c / nx), x = (int)(c - (long long)y * nx);
    int to = (int)c;
    if (x > 0 && y > 0 && x < nx - 1 && y < ny - 1) {
      K best = FK::of(a.h[c]);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int n = (int)c + nbr_off(k, nx);
        const K kn = FK::of(a.h[n]);
        if (kn < best) {
          best = kn;
          to = n;
        }
      }
    }
    a.ptr[c] = to;
  }
  if (!grid_barrier(a.st, G)) return;
  // pointer jumping until every pointer names its chain's end (chains are
  // strictly descending, so they end; in-place jumps only shorten them)
  for (int j = 0;; ++j) {
    bool moved = false;
    for (long long c = gtid; c < N; c += gstride) {
      const int p = __ldcg(a.ptr + c);
      const int pp = __ldcg(a.ptr + p);
      if (pp != p) {
        __stcg(a.ptr + c, pp);
        moved = true;
      }
    }
    if (__syncthreads_or(moved) && threadIdx.x == 0) a.fs->jump[j % 3] = 1;
    if (!grid_barrier(a.st, G)) return;
    if (lead) a.fs->jump[(j + 2) % 3] = 0;
    if (ld_volatile(&a.fs->jump[j % 3]) == 0) break;
    if (j >= 64) {  // a chain of 2^64 cells: cannot happen
      set_error(a.st, kErrInval);
      return;
    }
  }
  // w = h where the chain ends on the perimeter, +inf in the basins of
  // interior pits and flats; their tiles are dirty for the first round
  for (long long c = gtid; c < N; c += gstride) {
    const int e = __ldcg(a.ptr + c);
    const int ey = e / nx, ex = e - ey * nx;
    const bool drains = ex == 0 || ey == 0 || ex == nx - 1 || ey == ny - 1;
    a.w[c] = drains ? FK::of(a.h[c]) : FK::kInf;
    if (!drains) {
      const int y = (int)(c / nx), x = (int)(c - (long long)y * nx);
      a.dirty[(y / kFT) * a.tiles_x + x / kFT] = 1;
    }
  }
  if (!grid_barrier(a.st, G)) return;
  int r = 0;
  for (; r < a.max_rounds; ++r) {
    uint8_t* cur = a.dirty + (size_t)(r & 1) * a.ntiles;
    uint8_t* nxt = a.dirty + (size_t)((r + 1) & 1) * a.ntiles;
    for (;;) {
      int t = 0, d = 0;
      if (lane == 0) {
        t = atomicAdd(&a.fs->claim[r % 3], 1);
        if (t < a.ntiles) {
          d = *(volatile uint8_t*)(cur + t);
          if (d) cur[t] = 0;  // cleared for its use as the next round's array
        }
      }
      t = __shfl_sync(0xffffffffu, t, 0);
      d = __shfl_sync(0xffffffffu, d, 0);
      if (t >= a.ntiles) break;
      if (!d) continue;
      const int res = fill_tile(a, t, sW, sH, lane);
      if (res != 0 && lane < 9) {
        // the eight neighbour tiles (lanes 0-7), and the tile itself if it
        // did not settle (lane 8)
        const int ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
        const int tiles_y = a.ntiles / a.tiles_x;
        const int k = lane < 4 ? lane : lane + 1;  // skip the centre (4) for lanes 0-7
        const int nty = lane == 8 ? ty : ty + k / 3 - 1;
        const int ntx = lane == 8 ? tx : tx + k % 3 - 1;
        const bool want = lane < 8 || res == 2;
        if (want && ntx >= 0 && ntx < a.tiles_x && nty >= 0 && nty < tiles_y) {
          nxt[nty * a.tiles_x + ntx] = 1;
          a.fs->mark[r % 3] = 1;
        }
      }
    }
    if (!grid_barrier(a.st, G)) return;
    if (lead) {
      a.fs->claim[(r + 2) % 3] = 0;
      a.fs->mark[(r + 2) % 3] = 0;
    }
    if (ld_volatile(&a.fs->mark[r % 3]) == 0) break;  // the same answer on every block
  }
  if (r == a.max_rounds) {
    set_error(a.st, kErrTimeout);
    return;
  }
  if (lead) a.fs->rounds = r + 1;
  // (read from L2: this thread's own initial stores may still sit in L1)
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N;
       c += (long long)G * blockDim.x)
    a.h[c] = FK::value(__ldcg(a.w + c));
}

template <typename HT>
int fill_launch_typed(lem_ctx* c) {
  const int tiles_x = (c->p.nx + kFT - 1) / kFT, tiles_y = (c->p.ny + kFT - 1) / kFT;
  const int ntiles = tiles_x * tiles_y;
  const size_t smem = (size_t)fill_warps<HT>() * fill_warp_bytes<HT>();
  const int threads = fill_warps<HT>() * 32;
  cudaError_t e = cudaSuccess;
  if (!c->fill_w) {
    e = cudaFuncSetAttribute((const void*)&fill_kernel<HT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nsm = 0, per_sm = 0;
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)&fill_kernel<HT>,
                                                        threads, smem);
    if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) c->fill_grid = nsm * per_sm;
    if (e == cudaSuccess) e = cudaMalloc(&c->fill_w, (size_t)c->N * sizeof(HT));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->fill_dirty, 2 * (size_t)ntiles);
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->fill_ptr, (size_t)c->N * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->fill_state, sizeof(FillState));
    if (e != cudaSuccess) {
      cudaFree(c->fill_w);
      cudaFree(c->fill_dirty);
      cudaFree(c->fill_state);
      cudaFree(c->fill_ptr);
      c->fill_ptr = nullptr;
      c->fill_w = nullptr;
      c->fill_dirty = nullptr;
      c->fill_state = nullptr;
      return e == cudaErrorMemoryAllocation ? LEM_ENOMEM : LEM_ECUDA;
    }
  }
  // no tile is dirty until the kernel marks the basins' tiles; counters
  // start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(c->fill_dirty, 0, 2 * (size_t)ntiles, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->fill_state, 0, sizeof(FillState), c->stream);
  FillArgs<HT> a;
  a.nx = c->p.nx;
  a.ny = c->p.ny;
  a.tiles_x = tiles_x;
  a.ntiles = ntiles;
  // a round settles at least one more tile crossing of every cell's least
  // flood path, and a path crosses fewer tile borders than it has cells:
  // N + 2 rounds is a bound that a correct flood never reaches
  a.max_rounds = c->N + 2;
  a.h = (HT*)c->h;
  a.w = (typename FillKey<HT>::K*)c->fill_w;
  a.dirty = c->fill_dirty;
  a.ptr = c->fill_ptr;
  a.fs = (FillState*)c->fill_state;
  a.st = c->st;
  void* args[] = {&a};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void*)&fill_kernel<HT>, dim3(c->fill_grid),
                                    dim3(threads), args, smem, c->stream);
  if (e == cudaSuccess) return LEM_OK;
  return e == cudaErrorMemoryAllocation ? LEM_ENOMEM : LEM_ECUDA;
}

}  // namespace lem

// The flood on the context's bound elevations (allocates its scratch on
// the first call); asynchronous on the context's stream.
int lem_fill_launch(lem_ctx* c) {
  return c->p.dtype == LEM_F64 ? lem::fill_launch_typed<double>(c)
                               : lem::fill_launch_typed<float>(c);
}

extern "C" {

int lem_fill(lem_ctx* c) {
  if (!c) return LEM_EINVAL;
  if (!c->h) return LEM_ESTATE;
  const int rc = lem_fill_launch(c);
  if (rc != LEM_OK) return rc;
  if (!c->frozen) c->rec_valid = c->lev_valid = c->acc_valid = false;
  return LEM_OK;
}

int lem_set_fill(lem_ctx* c, int on) {
  if (!c || (on != 0 && on != 1)) return LEM_EINVAL;
  c->fill_on = on;
  return LEM_OK;
}

int lem_fill_stats(lem_ctx* c, int64_t* stats) {
  if (!c || !stats) return LEM_EINVAL;
  for (int i = 0; i < 4; ++i) stats[i] = 0;
  if (!c->fill_state) return LEM_OK;
  lem::FillState f;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMemcpy(&f, c->fill_state, sizeof(f), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LEM_ECUDA;
  stats[0] = f.rounds;
  stats[1] = f.visits;
  stats[2] = (int64_t)f.passes;
  stats[3] = f.unsettled;
  return LEM_OK;
}

}  // extern "C"
