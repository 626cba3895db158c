// lem_tiles.cuh -- Algs 3-6 of one time step on warp-private forests.
//
// Included by lem_step_kernel.cuh after the phase functions it builds on.
//
// The grid is cut into tiles of kTileW x tile_h<HT>() cells.  A warp takes one
// tile at a time and handles every tree rooted at one of the tile's cells
// without receiver (level 0 of Alg 3): it grows their breadth-first levels
// (Alg 3), pushes cell counts from the deepest level up (Alg 4) and erodes
// from level 0 up (Algs 5-6), entirely in its own slice of shared memory and
// with warp barriers only.  Trees are disjoint, so warps never touch the same
// cell and need no synchronisation with one another -- the paper's private
// queues ("Independent Parallelism", RB+PQ) at warp granularity, with the
// queue held on chip.  The donor masks (Alg 2) come from the codes pass.
//
// A forest that outgrows the warp's slice (kCap entries or kTileLv levels)
// is abandoned before anything is written; its tile goes to the block tier,
// which runs the same trees on a block-private queue in global memory with
// block barriers (private_forest).  A block whose tier outgrows its queue
// share hands the roots to the device tier: device-wide levels after a grid
// barrier (phase_global_levels and friends).  Every tier applies the same
// per-cell arithmetic, so the elevations do not depend on which tier ran.
#pragma once

namespace lem {

static_assert(2 * (kTileLv + 1) <= kTileLvBytes, "level offsets fit");

// One warp's forest in shared memory.  Entry j: cell c[j]; the word pd[j]
// = cell count << 16 | parent entry (the entry of its receiver) << 4 |
// receiver code (0..7 for levels >= 1, 8 or 9 at level 0); and v[j], the
// cell's elevation, copied in asynchronously when the entry is created and
// replaced by the new elevation when the entry is eroded.
template <typename HT>
struct TileQ {
  static constexpr int kHead = kTileLvBytes;
  static constexpr int kEntryBytes = (int)sizeof(HT) + 4 + 4;
  static constexpr int kCap = ((kWarpBytes - kHead) / kEntryBytes) & ~7;
  static_assert(kCap >= kTileW * tile_h<HT>(), "a tile's level 0 always fits");
  static_assert(kCap < (1 << 12), "parent index and count fit pd");
  static_assert(kHead % 16 == 0, "entry arrays stay aligned");
  unsigned short* lev;
  HT* v;
  int* c;
  unsigned* pd;
  __device__ __forceinline__ explicit TileQ(unsigned char* base) {
    lev = reinterpret_cast<unsigned short*>(base);
    v = reinterpret_cast<HT*>(base + kHead);
    c = reinterpret_cast<int*>(base + kHead + sizeof(HT) * kCap);
    pd = reinterpret_cast<unsigned*>(base + kHead + (sizeof(HT) + 4) * kCap);
  }
};

// g_nth[m * 8 + r]: the position of the r-th lowest set bit (r = 0, 1, ...)
// of the 8-bit donor mask m, 0 where m has no such bit.  A window of Alg 3
// hands each lane one donor as "bit r of its parent's mask"; one lookup
// replaces clearing r bits one at a time.  One table per block, filled by
// fill_nth (all threads, then a block barrier) before the first forest.
static __shared__ unsigned char g_nth[256 * 8];
__device__ __forceinline__ void fill_nth(int t, int nthreads) {
  for (int i = t; i < 256 * 8; i += nthreads) {
    unsigned m = (unsigned)i >> 3;
    for (int r = 0; r < (i & 7); ++r) m &= m - 1u;
    g_nth[i] = (unsigned char)(m ? __ffs(m) - 1 : 0);
  }
}

// g_ptab[32 w + e]: warp w's start -> lane table of the current window of
// Alg 3 (the lane whose donors start at position e of the window's donor
// list), written and read between warp barriers.
static __shared__ unsigned char g_ptab[32 * 32];

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// A unit of warp-tier work: the trees rooted in all rows of a tile, or in
// one half of its rows (the last tiles of a step are split in two so that
// the warps finish closer together).  Packed as tile << 2 | part, part 0 =
// every row, 1 = rows [0, TH/2), 2 = rows [TH/2, TH).
__device__ __forceinline__ int tile_item(int tile, int part) { return tile << 2 | part; }
template <int TH>
__device__ __forceinline__ void item_rows(int item, int* tile, int* rlo, int* rhi) {
  const int part = item & 3;
  *tile = item >> 2;
  *rlo = part == 2 ? TH / 2 : 0;
  *rhi = part == 1 ? TH / 2 : TH;
}

// Level 0 of one tile as seen by lane `lane`: the row codes of its column,
// for rows [rlo, rhi).  Other rows and out-of-grid positions read as 0 (a
// cell with a receiver: never a root).
template <int TH>
__device__ __forceinline__ void tile_codes(const uint8_t* code, int tile, int rlo, int rhi,
                                           int tiles_x, int nx, int ny, int lane, int* cd, int* x,
                                           int* y0) {
  const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
  *x = tx * kTileW + lane;
  *y0 = ty * TH;
#pragma unroll
  for (int r = 0; r < TH; ++r) {
    const int y = *y0 + r;
    cd[r] = (*x < nx && y < ny && r >= rlo && r < rhi) ? code[(size_t)y * nx + *x] : 0;
  }
}

// Append the roots of work item `item` to the device tier's level 0
// (queue[0, n)).
template <int TH>
__device__ __forceinline__ void push_tile_roots_device(const uint8_t* code, int* queue,
                                                       int* dev_roots, int item, int tiles_x,
                                                       int nx, int ny, int lane) {
  int cd[TH], x, y0, tile, rlo, rhi;
  item_rows<TH>(item, &tile, &rlo, &rhi);
  tile_codes<TH>(code, tile, rlo, rhi, tiles_x, nx, ny, lane, cd, &x, &y0);
#pragma unroll
  for (int r = 0; r < TH; ++r) {
    const bool f = cd[r] >= kSink;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (bal == 0) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(dev_roots, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (f) queue[base + __popc(bal & ((1u << lane) - 1u))] = (y0 + r) * nx + x;
  }
}

// Erosion parameters of the warp tier, copied out of the kernel parameter
// once per tile so that stores to h do not force them to be reloaded.  All
// of a warp forest's counts are below kTableN: g always comes from a table.
template <typename HT, bool kNewton = false>
struct TileErode {
  const void* gtab;  // F/(1+F): double2 {F, g} (FP64) or float (FP32); diagonal at +tn
  int tn;            // counts tabulated (every warp-forest count is below it)
  const double* Uf;
  double Udt, dt;
  float Udt_f;
  // Alg 6 for a general slope exponent (kNewton): the {F, g} table (for
  // either elevation type), d^(1-n) for cardinal and diagonal receivers,
  // the exponent, the tolerance and the update limit
  const double2* Ftab;
  double dfac, dfacd, nexp, neps;
  int iters;
  // Alg 5: h + dt*U (the same operations as uplift_sink).  kField: U is the
  // per-cell field Uf (else the scalar Udt); the caller picks the form once
  // per forest, so the per-cell code carries no test of Uf.
  template <bool kField>
  __device__ __forceinline__ HT uplift(int c, HT hcur) const {
    if constexpr (sizeof(HT) == 8) {
      return __dadd_rn(hcur, kField ? __dmul_rn(Uf[c], dt) : Udt);
    } else {
      return __fadd_rn(hcur, kField ? (float)__dmul_rn(Uf[c], dt) : Udt_f);
    }
  }
  template <bool kField>
  __device__ __forceinline__ HT erode(int c, int k, unsigned count, HT hcur, HT hr) const {
    const int i = (nbr_diag(k) ? tn : 0) + (int)count;
    if constexpr (kNewton) {
      // the operations of erode_newton for a tabulated count
      const double h0 = (double)hcur + (kField ? __dmul_rn(Uf[c], dt) : Udt);
      const double F = Ftab[i].x * (nbr_diag(k) ? dfacd : dfac);
      return (HT)newton_solve(h0, (double)hr, F, nexp, neps, iters);
    } else if constexpr (sizeof(HT) == 8) {
      const double g = static_cast<const double2*>(gtab)[i].y;
      const double h0 = __dadd_rn(hcur, kField ? __dmul_rn(Uf[c], dt) : Udt);
      return __fma_rn(-g, __dsub_rn(h0, hr), h0);
    } else {
      const float g = static_cast<const float*>(gtab)[i];
      const float h0 = __fadd_rn(hcur, kField ? (float)__dmul_rn(Uf[c], dt) : Udt_f);
      return __fmaf_rn(-g, __fsub_rn(h0, hr), h0);
    }
  }
};


// What a warp forest reads: the grid, its codes and masks (Algs 1-2 done),
// the elevations it erodes and the erosion parameters.
template <typename HT, bool kNewton = false>
struct TileArgs {
  int nx, ny, tiles_x;
  DevState* st = nullptr;  // index checks of the LEM_DEBUG build report here
  const uint8_t* code;
  const uint8_t* mask;
  HT* h;
  TileErode<HT, kNewton> ero;
};

// Algs 3-6 on the trees rooted in work item `item` (tile_item), by one warp.
// off[k] is the address offset of neighbour k.  Returns the number of cells
// handled, or -1 if the forest does not fit (nothing was written).
template <typename HT, bool kNewton>
__device__ __forceinline__ int tile_forest(const TileArgs<HT, kNewton>& a, const TileQ<HT>& q,
                                           const int* off, int item, int lane) {
  using Q = TileQ<HT>;
  // the arguments used in the loops, held in registers (stores through other
  // pointers would otherwise force reloads)
  const int nx = a.nx, ny = a.ny, tiles_x = a.tiles_x;
  const uint8_t* const mask = a.mask;
  const uint8_t* const code = a.code;
  const HT* const h = a.h;
  // level 0: the item's cells without receiver, in row order.  The tile's
  // codes are read as 4-byte words (8 per row; lane l takes words l, l + 32,
  // ...), and one scan of the words' root counts (packed in 10-bit fields)
  // places every root.  In-grid codes are 0..9, so a root is a byte with
  // bit 3 set; bytes outside the grid or the item's rows read as 0.
  int n = 0;
  {
    const int tile = item >> 2, part = item & 3;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    constexpr int TH = tile_h<HT>();
    constexpr int kWords = TH * kTileW / 4 / 32;  // code words per lane
    static_assert(TH * kTileW % 128 == 0 && kWords <= 3, "whole words per lane, 10-bit fields");
    const int x0 = tx * kTileW, y0 = ty * TH;
    const int rlo = part == 2 ? TH / 2 : 0, rhi = part == 1 ? TH / 2 : TH;
    unsigned roots[kWords];
    int packed = 0;
#pragma unroll
    for (int i = 0; i < kWords; ++i) {
      const int jw = lane + 32 * i, r = jw >> 3, xq = x0 + 4 * (jw & 7), y = y0 + r;
      unsigned v = 0;
      if (r >= rlo && r < rhi && y < ny && xq < nx) {
        const uint8_t* p = code + (size_t)y * nx + xq;
        if (xq + 3 < nx && ((size_t)p & 3) == 0) {
          v = *reinterpret_cast<const unsigned*>(p);
        } else {
          for (int b = 0; b < 4 && xq + b < nx; ++b) v |= (unsigned)p[b] << (8 * b);
        }
      }
      roots[i] = v & 0x08080808u ? v : 0u;  // keep the codes of words with a root
      packed |= __popc(v & 0x08080808u) << (10 * i);
    }
    int incl = packed;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - packed;
#pragma unroll
    for (int i = 0; i < kWords; ++i) {
      const unsigned v = roots[i];
      unsigned rb = v & 0x08080808u;
      int pos = n + ((excl >> (10 * i)) & 1023);
      const int jw = lane + 32 * i;
      const int cw = (y0 + (jw >> 3)) * nx + x0 + 4 * (jw & 7);
      while (rb) {
        const int bit = __ffs(rb) - 1;  // 3, 11, 19 or 27
        rb &= rb - 1;
        const int c = cw + (bit >> 3);
        q.c[pos] = c;
        q.pd[pos] = (v >> (bit - 3)) & 0xFFu;
        cp_async_elem(q.v + pos, h + c, true);
        ++pos;
      }
      n += (tot >> (10 * i)) & 1023;
    }
  }
  if (lane == 0) {
    q.lev[0] = 0;
    q.lev[1] = (unsigned short)n;
  }
  __syncwarp();
  // Alg 3 as one first-in first-out sweep: each window takes the next 32
  // entries, whatever their levels, and appends their donors (k order per
  // entry, entries in queue order), so the queue stays in level order.  The
  // window that holds the first entry of level L ends level L+1's
  // predecessors: level L+1 starts after the donors of the entries before it.
  // The next window's entries that already exist when a window starts (most
  // of them: the queue usually runs a window ahead) have their cell and mask
  // loaded then, so the mask load overlaps this window's work instead of
  // heading the next window's dependency chain.  pre: entries below it were
  // prefetched into (cn, mn) for the lane's entry of the coming window.
  int head = 0, tail = n, L = 1, B = n;  // B: first entry of level L
  int cn = 0, mn = 0, pre = 0;
  while (head < tail) {
    const int w = min(32, tail - head);
    const int j = head + lane;
    int c = 0, msk = 0;
    if (lane < w) {
      if (j < pre) {
        c = cn;
        msk = mn;
      } else {
        c = q.c[j];
        msk = mask[c];
      }
    }
    pre = tail;
    if (j + w < tail) {
      cn = q.c[j + w];
      mn = mask[cn];
    }
    const int k = __popc(msk);
    int incl = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    if (tail + tot > Q::kCap) {
      cp_async_wait_all();  // no copy may land in the slice after we leave
      return -1;
    }
    if (B >= head && B < head + w) {
      const int before = B - head;  // lanes of level L-1 in this window
      const int sb = __shfl_sync(0xffffffffu, incl, before > 0 ? before - 1 : 0);
      if (L >= kTileLv) {
        cp_async_wait_all();
        return -1;
      }
      ++L;
      B = tail + (before > 0 ? sb : 0);
      if (lane == 0) q.lev[L] = (unsigned short)B;
    }
    // the window's tot donors, one per lane: donor e belongs to the lane s
    // with excl(s) <= e < incl(s), as its (e - excl(s))-th set bit.  The
    // first 32 (usually all of them): the lanes with donors are the ones
    // whose start excl(s) is the largest start <= e, so a bitmap of the starts
    // and a start -> lane table give s in a few instructions
    if (tot > 0) {
      unsigned char* const ptab = g_ptab + (threadIdx.x >> 5) * 32;
      const int ex = incl - k;
      const bool starts = k > 0 && ex < 32;
      if (starts) ptab[ex] = (unsigned char)lane;
      const unsigned sb = __reduce_or_sync(0xffffffffu, starts ? 1u << ex : 0u);
      __syncwarp();
      // bit 0 is set (the first lane with donors starts at 0), so p >= 0
      const int p = 31 - __clz(sb & (0xFFFFFFFFu >> (31 - lane)));
      const int s = ptab[p];
      const int pm = __shfl_sync(0xffffffffu, msk, s);
      const int pc = __shfl_sync(0xffffffffu, c, s);
      if (lane < tot) {
        const int kk = g_nth[pm * 8 + (lane - p)];
        const int pos = tail + lane;
        const int cc = pc + off[kk];
        if (in_bounds(a.st, pos, Q::kCap) && in_bounds(a.st, cc, (long long)nx * ny)) {
          q.c[pos] = cc;
          q.pd[pos] = (1u << 16) | ((unsigned)(head + s) << 4) | (unsigned)(7 - kk);
          cp_async_elem(q.v + pos, h + cc, true);
        }
      }
    }
    // donors 32 and up: s by a binary search over the inclusive counts
    for (int e0 = 32; e0 < tot; e0 += 32) {
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
        // the (e - pex)-th set bit of the parent's mask (it has more bits)
        const int kk = g_nth[pm * 8 + (e - pex)];
        const int pos = tail + e;
        const int cc = pc + off[kk];
        if (!in_bounds(a.st, pos, Q::kCap) || !in_bounds(a.st, cc, (long long)nx * ny)) continue;
        q.c[pos] = cc;
        q.pd[pos] = (1u << 16) | ((unsigned)(head + s) << 4) | (unsigned)(7 - kk);
        cp_async_elem(q.v + pos, h + cc, true);
      }
    }
    tail += tot;
    head += w;
    __syncwarp();
  }
  // levels 0 .. L-1; q.lev[L] == tail
  // Alg 4: each entry adds its final count to its parent's, deepest level
  // first; level 1 has no eroding parent to feed
  for (int l = L - 1; l >= 2; --l) {
    const int l0 = q.lev[l], l1 = q.lev[l + 1];
    for (int jj = l0 + lane; jj < l1; jj += 32) {
      const unsigned w = q.pd[jj];
      atomicAdd(&q.pd[(w >> 4) & 0xFFFu], w & 0xFFFF0000u);
    }
    __syncwarp();
  }
  cp_async_wait_all();  // every entry's elevation has arrived
  __syncwarp();
  const TileErode<HT, kNewton> ero = a.ero;
  HT* const hh = a.h;
  auto erode_levels = [&](auto field) {
    constexpr bool kField = decltype(field)::value;
    // Alg 5 on level 0: pits are uplifted, the perimeter stays
    for (int jj = lane; jj < n; jj += 32) {
      if ((q.pd[jj] & 15u) == (unsigned)kSink) {
        const int c = q.c[jj];
        const HT hc = ero.template uplift<kField>(c, q.v[jj]);
        hh[c] = hc;
        q.v[jj] = hc;
      }
    }
    __syncwarp();
    // Alg 6 from level 1 up: the receiver's new elevation is the parent's v
    for (int l = 1; l < L; ++l) {
      const int l0 = q.lev[l], l1 = q.lev[l + 1];
      for (int jj = l0 + lane; jj < l1; jj += 32) {
        const int c = q.c[jj];
        const unsigned pd = q.pd[jj];
        const HT hn = ero.template erode<kField>(c, (int)(pd & 15u), pd >> 16, q.v[jj],
                                                 q.v[(pd >> 4) & 0xFFFu]);
        if (in_bounds(a.st, c, (long long)nx * ny)) hh[c] = hn;
        q.v[jj] = hn;
      }
      __syncwarp();
    }
  };
  if (ero.Uf != nullptr) {
    erode_levels(Flag<true>{});
  } else {
    erode_levels(Flag<false>{});
  }
  return tail;
}

// The block tier: level 0 = the roots of this block's nov overflowed tiles
// (s.ovf_tiles).  Returns the number of cells handled, or 0 after handing
// the roots to the device tier when the block's queue cannot hold them.
template <typename HT, typename CT, bool kNewton>
__device__ __noinline__ int block_tier(const StepArgs<HT, CT>& a, Shared& s, int nov,
                                       int* dev_roots) {
  const int b = blockIdx.x, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int nx = a.nx, ny = a.ny;
  int* pq = a.pq + (size_t)b * a.pcap;
  uint8_t* pqm = a.pqm + (size_t)b * a.pcap;
  uint8_t* pqk = a.pqk + (size_t)b * a.pcap;
  constexpr int TH = tile_h<HT>();
  if (a.jt != nullptr && ld_volatile(&a.st->jump_hint) != 0) {
    // the last device tier was deep: these trees go straight to it
    for (int i = w; i < nov; i += kWarps)
      push_tile_roots_device<TH>(a.code, a.queue, dev_roots, s.ovf_tiles[i], a.tiles_x, nx, ny,
                                 lane);
    return 0;
  }
  for (int i = w; i < nov; i += kWarps) {
    int cd[TH], x, y0, tile, rlo, rhi;
    item_rows<TH>(s.ovf_tiles[i], &tile, &rlo, &rhi);
    tile_codes<TH>(a.code, tile, rlo, rhi, a.tiles_x, nx, ny, lane, cd, &x, &y0);
#pragma unroll
    for (int r = 0; r < TH; ++r) {
      const bool f = cd[r] >= kSink;
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (bal == 0) continue;
      int base = 0;
      if (lane == 0) base = atomicAdd(&s.n0, __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      const int pos = base + __popc(bal & ((1u << lane) - 1u));
      if (f && pos < a.pcap) {
        const int c = (y0 + r) * nx + x;
        pq[pos] = c;
        pqk[pos] = (uint8_t)cd[r];
        pqm[pos] = a.mask[c];
      }
    }
  }
  __syncthreads();
  const int n0 = s.n0;
  const int done = (n0 <= a.pcap) ? private_forest<HT, CT, kNewton>(a, s, n0) : -1;
  if (done >= 0) return done;
  for (int i = w; i < nov; i += kWarps)
    push_tile_roots_device<TH>(a.code, a.queue, dev_roots, s.ovf_tiles[i], a.tiles_x, nx, ny,
                               lane);
  return 0;
}

// The warp tier of one step.  Work items (tiles, or halves of the last
// tiles) are claimed from a device-wide counter; a whole tile whose forest
// does not fit a warp is retried as its two halves, and an item that still
// does not fit is appended to the device-wide overflow list ovf[] (counter
// *n_ovf) for the block tier.  The cells handled are added to *covered and
// to the warp tier's total.
template <typename HT, typename CT, bool kNewton>
__device__ __noinline__ void phase_tiles(const StepArgs<HT, CT>& a, Shared& s, int* tiles_next,
                                         int* n_ovf, int* ovf, int* covered) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  const TileQ<HT> q(dyn_smem + w * kWarpBytes);
  if (t < 8) s.off[t] = nbr_off(t, a.nx);
  fill_nth(t, kBD);
  __syncthreads();
  TileArgs<HT, kNewton> ta;
  ta.nx = a.nx;
  ta.ny = a.ny;
  ta.tiles_x = a.tiles_x;
  ta.st = a.st;
  ta.code = a.code;
  ta.mask = a.mask;
  ta.h = a.h;
  if constexpr (sizeof(HT) == 8) {
    ta.ero.gtab = a.Ftab;
  } else {
    ta.ero.gtab = a.gtab;
  }
  ta.ero.tn = kTableN;
  ta.ero.Uf = a.Uf;
  ta.ero.Udt = a.Udt;
  ta.ero.dt = a.dt;
  ta.ero.Udt_f = a.Udt_f;
  if constexpr (kNewton) {
    ta.ero.Ftab = a.Ftab;
    ta.ero.dfac = a.dfac;
    ta.ero.dfacd = a.dfacd;
    ta.ero.nexp = a.nexp;
    ta.ero.neps = a.neps;
    ta.ero.iters = a.newton_iters;
  }
  long long mine = 0;
  // work items are claimed one at a time from a device-wide counter, the
  // next claim issued before the current item is processed.  Claims below
  // T - S are whole tiles; the last S tiles (one per four warps of the
  // grid) are claimed as halves, so the last claims are half as long.
  // Lane 0 maps a claim to its item (-1: none left).
  const auto item_of = [&](int claim) {
    const int T = a.ntiles;
    const int S = a.half_tiles ? T : min(T, (int)gridDim.x * (kWarps / 4)), TF = T - S;
    if (claim >= T + S) return -1;
    return claim < TF ? tile_item(claim, 0)
                      : tile_item(TF + ((claim - TF) >> 1), 1 + ((claim - TF) & 1));
  };
  int item = 0;
  if (lane == 0) item = item_of(atomicAdd(tiles_next, 1));
  item = __shfl_sync(0xffffffffu, item, 0);
  // pend: the second half of a split tile, run after the first; the next
  // claim is taken once per claimed item (all warp-uniform)
  int next = -1, pend = -1;
  bool claimed = false;
  while (item >= 0) {
    if (!claimed) {
      int nc = 0;
      if (lane == 0) nc = item_of(atomicAdd(tiles_next, 1));
      next = __shfl_sync(0xffffffffu, nc, 0);
      claimed = true;
    }
    const int r = tile_forest(ta, q, s.off, item, lane);
    const int cur = item;
    if (r >= 0) {
      mine += r;
    } else if ((cur & 3) == 0) {
      // a whole tile whose forest did not fit (nothing was written): its
      // two halves hold fewer roots each and usually fit
      item = cur | 1;
      pend = cur | 2;
      continue;
    } else if (lane == 0) {
      ovf[atomicAdd(n_ovf, 1)] = cur;
    }
    if (pend >= 0) {
      item = pend;
      pend = -1;
      continue;
    }
    item = next;
    claimed = false;
  }
  // per-warp totals (lane 0's count is the warp's)
  if (lane == 0) s.wcount[w] = (int)mine;
  __syncthreads();
  trace_point(a.st, kTrLocal + 4);
  if (t == 0) {
    long long by_warps = 0;
    for (int i = 0; i < kWarps; ++i) by_warps += s.wcount[i];
    atomicAdd(covered, (int)by_warps);
    atomicAdd(&a.st->tier_cells[0], (unsigned long long)by_warps);
  }
}

// The block tier of one step, after a grid barrier: the n overflowed items
// of the list ovf[] are owned by block (tile index mod grid size) -- a rule
// that does not depend on which warp found them, so each block's forest,
// and whether it fits, is the same in every run.  A block that owns more
// than kOvfCap items hands all their roots to the device tier.
template <typename HT, typename CT, bool kNewton>
__device__ __noinline__ void phase_block_tier(const StepArgs<HT, CT>& a, Shared& s, int n,
                                              const int* ovf, int* dev_roots, int* covered) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int b = blockIdx.x, G = (int)gridDim.x;
  constexpr int TH = tile_h<HT>();
  if (t == 0) {
    s.n_ovf = 0;
    s.n0 = 0;
  }
  if (t < 8) s.off[t] = nbr_off(t, a.nx);
  __syncthreads();
  for (int i = t; i < n; i += kBD) {
    const int it = __ldcg(ovf + i);
    if ((it >> 2) % G == b) {
      const int k = atomicAdd(&s.n_ovf, 1);
      if (k < kOvfCap) s.ovf_tiles[k] = it;
    }
  }
  __syncthreads();
  const int nov = s.n_ovf;
  long long by_block = 0;
  if (nov > kOvfCap) {
    for (int i = t >> 5; i < n; i += kWarps) {
      const int it = __ldcg(ovf + i);
      if ((it >> 2) % G == b)
        push_tile_roots_device<TH>(a.code, a.queue, dev_roots, it, a.tiles_x, a.nx, a.ny, lane);
    }
  } else if (nov > 0) {
    by_block = block_tier<HT, CT, kNewton>(a, s, nov, dev_roots);
  }
  (void)w;
  trace_point(a.st, kTrLocal + 5);
  if (t == 0 && by_block > 0) {
    atomicAdd(covered, (int)by_block);
    atomicAdd(&a.st->tier_cells[1], (unsigned long long)by_block);
  }
}

}  // namespace lem
