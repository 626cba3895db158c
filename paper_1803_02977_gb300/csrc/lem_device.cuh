// lem_device.cuh -- device-side building blocks shared by the library's
// kernels: neighbour geometry, the status word, a bounded grid barrier and a
// block-wide scan.  sm_103a only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lem {

// Receiver code of a cell: 0..7 = neighbour k (0=NW 1=N 2=NE 3=W 4=E 5=SW
// 6=S 7=SE, ascending address order); 8 = interior cell without receiver
// (a pit: uplifted, not eroded); 9 = perimeter cell (fixed base level).
constexpr int kSink = 8;
constexpr int kEdge = 9;
__host__ __device__ __forceinline__ bool no_receiver(int code) { return code >= kSink; }

// Erosion factors are tabulated for counts below this bound.
constexpr int kTableN = 1 << 16;

// Status codes written into the device status word (same values as lem.h).
constexpr int kErrInval = -1;
constexpr int kErrTimeout = -4;
constexpr int kErrBounds = -7;

// Index checks of the LEM_DEBUG build (the library compiled with -DLEM_DEBUG,
// liblem_debug.so): every guarded access checks its index against the array
// it touches; one out of range records kErrBounds and is skipped -- never a
// trap, so the kernel keeps its barriers and the context stays usable.  In
// the regular build the checks compile away.
#ifdef LEM_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif

// Phase bits of the persistent step kernel.
constexpr int kPhRec = 1;     // Alg 1 receivers + Alg 2 donor masks + level 0
constexpr int kPhLev = 2;     // Alg 3 breadth-first levels
constexpr int kPhAcc = 4;     // Alg 4 accumulation
constexpr int kPhEro = 8;     // Alg 5 + Alg 6
constexpr int kPhAll = 15;
// Algs 3-6 on warp-private forests in shared memory, with block-private and
// device-wide tiers for trees that do not fit (lem_step's default form).
constexpr int kPhTiles = 32;

__host__ __device__ __forceinline__ int nbr_dx(int k) {
  return (k == 0 || k == 3 || k == 5) ? -1 : ((k == 2 || k == 4 || k == 7) ? 1 : 0);
}
__host__ __device__ __forceinline__ int nbr_dy(int k) { return k < 3 ? -1 : (k < 5 ? 0 : 1); }
__host__ __device__ __forceinline__ bool nbr_diag(int k) {
  return k == 0 || k == 2 || k == 5 || k == 7;
}
__host__ __device__ __forceinline__ int nbr_off(int k, int nx) { return nbr_dy(k) * nx + nbr_dx(k); }

// Double nearest 1/sqrt(2), the diagonal slope weight (dist = dx*sqrt(2)).
constexpr double kInvSqrt2 = 0.70710678118654752440;
// Double nearest sqrt(2).
constexpr double kSqrt2 = 1.41421356237309504880;

// Global state of one context: grid-barrier words, sticky status, and the
// hand-off words of the single-block narrow-level mode.
struct DevState {
  unsigned int bar_count;
  unsigned int bar_gen;
  int err;
  int nlevels;
  int bfs_lo, bfs_hi, bfs_level, bfs_done;
  unsigned long long wait_limit_ns;
  int selftest_flag;  // never written by anyone: the self-test waits on it
  int trace_cap;      // capacity of trace (entries); 0 = tracing off
  int trace_n;        // entries written since the last read
  unsigned long long* trace;  // pairs {globaltimer ns, tag}
  int private_steps;     // steps completed without device-wide levels
  int global_steps;      // steps that needed device-wide levels
  // per-step words of the tiered step, double-buffered by step parity:
  // roots handed to the device tier, cells handled by all tiers
  int dev_roots[2];
  int covered[2];
  int tiles_next[2];  // warp-tier tiles claimed (zero between launches)
  int ovf_count[2];   // warp-tier items that did not fit (listed for the block tier)
  unsigned long long tier_cells[3];  // cells handled by warp, block, device tier
  // the device tier's pointer-jumping form (lem_jump.cuh)
  int jump_epoch;        // stamp of the latest jumping step (root marks)
  int jump_vote[3];      // per-round change votes
  int jump_hint;         // the last device tier was deep: jump at once
  int jump_rounds;       // erosion rounds of the latest jumping step
  int jump_steps;        // steps whose device tier jumped
  unsigned long long jump_step_cells;  // eroding cells of the latest jumping step
};

// Trace tags: phase in the high half, level (or 0) in the low half.
enum TraceTag : int {
  kTrStart = 1 << 16,     // kernel entered, step begins
  kTrCodes = 2 << 16,     // receiver codes done (barrier passed)
  kTrLevel0 = 3 << 16,    // donor masks and level 0 done
  kTrBfsWide = 4 << 16,   // one wide breadth-first level done
  kTrBfsNarrow = 5 << 16, // a run of narrow levels done by block 0
  kTrAccWide = 6 << 16,
  kTrAccNarrow = 7 << 16,
  kTrUplift = 8 << 16,
  kTrEroWide = 9 << 16,
  kTrEroNarrow = 10 << 16,
  kTrPrivBfs = 11 << 16,    // all blocks' private queues built (barrier passed)
  kTrPrivAcc = 12 << 16,    // block 0 finished its private accumulation
  kTrPrivEro = 13 << 16,    // block 0 finished its private erosion
  kTrStepEnd = 14 << 16,    // end-of-step barrier passed
  kTrLocal = 15 << 16,      // block 0 reached the next barrier (low half: which)
  kTrTilesEnd = 16 << 16,   // warp and block tiers done on every block (barrier passed)
  kTrJumpTour = 17 << 16,   // pointer-jumping tier: tour links built
  kTrJumpRank = 18 << 16,   // one list-ranking round (low half: round)
  kTrJumpInit = 19 << 16,   // counts, factors and first affine maps
  kTrJumpErode = 20 << 16,  // one erosion-jumping round (low half: round)
  kTrBlockEnd = 21 << 16,   // block tier done on every block (barrier passed)
};

// Record a timestamp (block 0, thread 0 only; no-op when tracing is off).
__device__ __forceinline__ void trace_point(DevState* st, int tag) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && st->trace_cap > 0) {
    const int i = st->trace_n;
    if (i < st->trace_cap) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      st->trace[2 * i] = t;
      st->trace[2 * i + 1] = (unsigned long long)(unsigned)tag;
    }
    st->trace_n = i + 1;
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_error(DevState* st, int code) { atomicCAS(&st->err, 0, code); }

// True if 0 <= i < n; in the LEM_DEBUG build, false (with kErrBounds
// recorded) otherwise.  The regular build always answers true.
__device__ __forceinline__ bool in_bounds(DevState* st, long long i, long long n) {
  if constexpr (kDebugChecks) {
    if (i < 0 || i >= n) {
      if (st) set_error(st, kErrBounds);
      return false;
    }
  }
  return true;
}


// Device-wide barrier for a co-resident (cooperative) grid.  Thread 0 of each
// block arrives on a counter; the last arrival resets it and advances the
// generation word that the others wait on.  Every wait is bounded by the
// context's wait limit and abandons early when another block has recorded an
// error; either way the function returns false and the caller must return.
__device__ __forceinline__ bool grid_barrier(DevState* st, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned gen = ld_acquire(&st->bar_gen);
    __threadfence();
    unsigned arrived = atomicAdd(&st->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      unsigned long long t0 = global_ns();
      unsigned it = 0;
      while (ld_acquire(&st->bar_gen) == gen) {
        if ((++it & 31u) == 0) {
          if (ld_volatile(&st->err) != 0) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > st->wait_limit_ns) {
            set_error(st, kErrTimeout);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Exclusive block-wide scan of one int per thread; *total receives the sum.
// scratch must hold BD/32 ints of shared memory.  Contains __syncthreads.
template <int BD>
__device__ __forceinline__ int block_exclusive_scan(int v, int* total, int* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = (lane < BD / 32) ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < BD / 32) scratch[lane] = s;
  }
  __syncthreads();
  int prefix = (w > 0) ? scratch[w - 1] : 0;
  *total = scratch[BD / 32 - 1];
  __syncthreads();
  return prefix + x - v;
}

template <int BD>
__device__ __forceinline__ long long block_sum(long long v, long long* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  long long s = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < BD / 32; ++i) s += scratch[i];
    scratch[0] = s;
  }
  __syncthreads();
  s = scratch[0];
  __syncthreads();
  return s;
}

}  // namespace lem
