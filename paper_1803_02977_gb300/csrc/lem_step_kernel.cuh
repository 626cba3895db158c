// lem_step_kernel.cuh -- the persistent cooperative kernel that runs the
// per-timestep method of Barnes (arXiv:1803.02977), Section "The Algorithm",
// Algorithms 1-6, on one GB300.
//
// One launch covers nsteps steps of one of two forms (phase bits):
//  * tiered (lem_step, kPhTiles): Algs 1-2 as a TMA-staged register stencil
//    over strips of the grid (phase_codes), a grid barrier, then Algs 3-6 on
//    warp-private tile forests in shared memory (lem_tiles.cuh) -- the
//    paper's private queues ("Independent Parallelism", RB+PQ) at warp
//    granularity -- with a block-private tier (private_forest) and a
//    device-wide tier for trees that do not fit, and a second grid barrier.
//  * device-wide (stage-by-stage calls, step mode 1, and the device tier):
//    Algs 1-2 with the cells without receiver compacted in ascending address
//    order (phase_receivers), then one breadth-first queue for the whole grid
//    with each level separated by a bounded grid barrier (the paper's
//    "for-parallel" level loops) and runs of narrow levels handled by block 0
//    alone.  This form produces the exported Queue and Levels in the
//    oracle's breadth-first order.
//
// Data layout (all in HBM, row-major grid order unless stated):
//   h      elevations (double or float), caller owned, updated in place
//   code   u8  receiver code per cell (0..7 neighbour k, 8 pit, 9 perimeter)
//   mask   u8  donor mask per cell: bit k set <=> neighbour k drains here
//   queue  i32 cells in breadth-first order (device-wide form)
//   levels i32 level offsets into queue, L+1 used
//   pq     i32 block-private queues, `pcap` entries per block
//   cnt    i32 or i64 cell counts (Alg 4's A in units of cells)
//
// FP64 on GB300 runs at about 1/70 of the FP32 rate, so the FP64 work per
// cell is kept small: receivers decide from the elevations' high words or
// bit patterns with FP32 slope margins and evaluate slopes in FP64 only for
// near ties (exact, see receiver_code_vals), and erosion uses the increment
// form of the implicit update with a tabulated F/(1+F) instead of a
// division (see erode_value).
#pragma once

#include "lem_device.cuh"

namespace lem {

// A TMA tensor descriptor (the driver's opaque 128-byte CUtensorMap), held
// in the kernel parameter so that each launch carries its own copy.
struct alignas(64) TmaDesc {
  unsigned long long w[16];
};

template <typename HT, typename CT>
struct StepArgs {
  int nx, ny, N;
  HT* h;
  const double* Uf;     // optional per-cell uplift rate
  double U, dt;         // scalar uplift rate, time step
  double Udt;           // U*dt, as Alg 5 forms it
  float Udt_f;          // U*dt rounded once to float
  double Kdt;           // K*dt
  double m, dx, dxd;    // area exponent, cardinal and diagonal distance
  double area_scale;
  uint8_t* code;
  uint8_t* mask;
  int* queue;
  int* levels;
  int* pq;              // block-private queues
  uint8_t* pqm;         // donor mask of each private-queue entry
  uint8_t* pqk;         // receiver code of each private-queue entry
  int* pqf;             // position of each private-queue entry's first donor
  CT* cntq;             // cell count of each private-queue entry (queue order)
  int pcap;             // entries per block in pq
  int tiles_x, ntiles;  // warp-tier tiles per row, in total
  int strip_rows;       // owned rows per strip of the codes pass (pick_strip_rows)
  int half_tiles;       // warp tier: every tile claimed as two half-height items
  int has_tmap;         // tmap describes h (else strips are staged element-wise)
  TmaDesc tmap;         // TMA descriptor of h: 2-D box of kStageCols x (strip_rows + 4)
  CT* cnt;
  const double2* Ftab;  // {F, F/(1+F)} for counts < kTableN: [0,N) cardinal, [N,2N) diagonal
  const float* gtab;    // F/(1+F) rounded to float, same layout
  DevState* st;
  int* partial;         // one int per block
  int phases;
  int nsteps;
  int frozen;           // receivers frozen: codes are inputs, not recomputed
  // Alg 6 for a general slope exponent (erode_newton): updates per cell, 0 for
  // the n = 1 closed form; exponent, tolerance, dx^n and (dx*sqrt2)^n
  int newton_iters = 0;
  double nexp = 1.0, neps = 0.0, dxn = 0.0, dxdn = 0.0;
  double dfac = 0.0, dfacd = 0.0;  // dx^(1-n) and (dx*sqrt2)^(1-n)
  // the device tier's pointer-jumping form (lem_jump.cuh): tour words (2 per
  // cell, reused as the first (A, B) buffer), the second (A, B) buffer, two
  // pointer buffers, a root stamp per cell; jt == nullptr turns it off.
  // jump_cap: breadth-first levels the device tier grows before it jumps.
  unsigned long long* jt = nullptr;
  double2* jab1 = nullptr;
  int* jp0 = nullptr;
  int* jp1 = nullptr;
  unsigned* jstamp = nullptr;
  int jump_cap = 0x7FFFFFFF;
  int priv_levels = 2048;  // levels a block-private queue may hold (<= kMaxPrivLevels)
};

constexpr int kCodeGuard = 16;     // 0xFF guard bytes on each side of the code array
constexpr int kBD = 1024;          // threads per block: one block per SM
constexpr int kWarps = kBD / 32;
constexpr int kItems = 4;          // items per thread per round in wide loops
// a device-wide level this small runs in block 0 alone, with block barriers
// instead of grid barriers (up to two rounds of the breadth-first emission,
// four cells per thread in the accumulation and erosion)
constexpr int kNarrowBfs = 2 * kBD;
constexpr int kNarrowSweep = kItems * kBD;
constexpr int kPItems = 8;         // entries per thread per round of a private level
constexpr int kStage = 16384;      // emitted entries staged in shared memory per round
constexpr int kMaxPrivLevels = 2048;  // level offsets a private queue may hold
constexpr int kOvfCap = 256;       // tiles a block keeps for its block tier
constexpr int kTileW = 32;         // warp-tier tile width: one column per lane
// warp-tier tile height: 8 rows with FP64 elevations, 12 with FP32 (whose
// queue entries are smaller, so a warp holds more of them)
template <typename HT>
__host__ __device__ constexpr int tile_h() {
  return sizeof(HT) == 4 ? 12 : 8;
}
// Shared memory per warp for its strip (Alg 1) and its forest (Algs 3-6).
// 32 slices of 6016 B and the block's static state stay within a 196 KB
// shared-memory carve-out, so 60 KB of the SM's 256 KB remain L1 (register
// spills and the scattered mask and table loads of the warp tier hit there);
// 7040 B slices needed the 228 KB carve-out and left 28 KB.  A multiple of
// 128 B, so that every slice can take a TMA box.
constexpr int kWarpBytes = 6016;
static_assert(kWarpBytes % 128 == 0, "warp slices start 128-byte aligned");
constexpr int kTileLv = 127;       // levels a warp forest may hold
constexpr int kTileLvBytes = 256;  // its level offsets, u16 [0, kTileLv]
// dynamic shared memory of the step kernel: the warps' forests, or (later in
// the step) the block tier's staging buffer
constexpr int kPlevOffset = kStage * (int)(sizeof(int) + 1);  // block tier: level offsets
constexpr int kBlockTierBytes = kPlevOffset + (kMaxPrivLevels + 1) * (int)sizeof(int);
constexpr int kDynSmem =
    kWarps * kWarpBytes > kBlockTierBytes ? kWarps * kWarpBytes : kBlockTierBytes;

// ---- Alg 1: receivers ----------------------------------------------------------

// Reference form: (h_c - h_n) * w in FP64 for all eight neighbours, strict
// '>' against an initial maximum of zero (lowest k wins ties).
static __device__ __noinline__ int receiver_code_slow(double hc, double h0, double h1, double h2,
                                               double h3, double h4, double h5, double h6,
                                               double h7) {
  const double hn[8] = {h0, h1, h2, h3, h4, h5, h6, h7};
  double smax = 0.0;
  int best = kSink;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double d = __dsub_rn(hc, hn[k]);
    const double s = nbr_diag(k) ? __dmul_rn(d, kInvSqrt2) : d;
    if (s > smax) {
      smax = s;
      best = k;
    }
  }
  return best;
}

// Bit-pattern view of non-negative finite elevations: for such values the
// unsigned order of the patterns is the numeric order.
template <typename HT> struct Bits;
template <> struct Bits<double> {
  using U = unsigned long long;
  static constexpr U kInf = 0x7FF0000000000000ull;
  static constexpr int kMant = 52;
  static constexpr int kExpBias = 0;  // steps counted in doubles
  __device__ static U of(double v) { return (U)__double_as_longlong(v); }
};
template <> struct Bits<float> {
  using U = unsigned int;
  static constexpr U kInf = 0x7F800000u;
  static constexpr int kMant = 23;
  static constexpr int kExpBias = 29;  // one float step spans 2^29 double steps
  __device__ static U of(float v) { return (U)__float_as_uint(v); }
};

// True if no runner-up value r (> m, < hc) can produce the same rounded FP64
// slope as the minimum m.  Two slopes fl(hc-a), or fl(fl(hc-a)*w), from a < b
// can only coincide when b - a < 4 ulp(hc); b - a is at least (number of
// representable steps from a to b) * (step at a), which bounds it from the
// bit patterns and exponents alone.
template <typename HT>
__device__ __forceinline__ bool no_rounding_merge(typename Bits<HT>::U m, typename Bits<HT>::U r,
                                                  typename Bits<HT>::U bc) {
  using B = Bits<HT>;
  if (r >= bc) return true;  // no second candidate below hc
  const int Ec = (int)(bc >> B::kMant);
  if (m == 0) {
    // a = 0 gives the exact difference hc; b must reach 4 ulp(hc)
    const int Er = (int)(r >> B::kMant);
    return Er >= 1 && Er >= Ec - 50;
  }
  const int Em = max((int)(m >> B::kMant), 1);
  const int sh = Ec - Em + 2 - B::kExpBias;
  if (sh <= 0) return true;  // any distinct pair is far enough apart
  if (sh > 62) return false;
  return (unsigned long long)(r - m) >= (1ull << sh);
}

// Alg 1 for one interior cell.  Exactly the reference form's result: the
// minimum elevation of each neighbour group (cardinal, diagonal) is found by
// comparing bit patterns (lowest k among equal values), and only the two
// group winners' slopes are evaluated in FP64 -- after checking that no other
// neighbour of the group could round to the same slope.  Cells where that
// check, or non-negative finiteness, fails take the reference form.
// FP64 elevations, first try: the same decision from the high 32-bit words
// of the values (sign, exponent, 20 mantissa bits), which order non-negative
// doubles like the values themselves.  A group's minimum is exact when its
// high word is unique in the group; no other member can round to the same
// slope when none has the next high word (then it lies more than 2^32 of the
// minimum's ulps above it) and the minimum lies at most 18 binades below h_c
// (so the 2^32 ulps between consecutive high words exceed 4 ulps of h_c).
// The two candidates' slopes are compared in FP32 from the high words
// (relative error below 2^-19 each), deciding when they differ by more than
// 2^-16 of h_c plus 2^-16 of the slopes.  Returns -1 when any of this does
// not hold (a minimum far below h_c, as the zero perimeter is for its
// interior neighbours, included).
__device__ __forceinline__ int receiver_code_hi_words(const unsigned hc, const unsigned* x) {
  unsigned worst = hc;
#pragma unroll
  for (int k = 0; k < 8; ++k) worst = max(worst, x[k]);
  const unsigned mC = min(min(x[1], x[3]), min(x[4], x[6]));
  const unsigned mD = min(min(x[0], x[2]), min(x[5], x[7]));
  const bool hasC = mC < hc, hasD = mD < hc;
  const unsigned eqC = (x[1] == mC ? 1u : 0u) | (x[3] == mC ? 2u : 0u) | (x[4] == mC ? 4u : 0u) |
                       (x[6] == mC ? 8u : 0u);
  const unsigned eqD = (x[0] == mD ? 1u : 0u) | (x[2] == mD ? 2u : 0u) | (x[5] == mD ? 4u : 0u) |
                       (x[7] == mD ? 8u : 0u);
  const bool nextC = x[1] == mC + 1 || x[3] == mC + 1 || x[4] == mC + 1 || x[6] == mC + 1;
  const bool nextD = x[0] == mD + 1 || x[2] == mD + 1 || x[5] == mD + 1 || x[7] == mD + 1;
  const bool badC = (eqC & (eqC - 1u)) != 0 || nextC || (hc >> 20) - (mC >> 20) > 18u;
  const bool badD = (eqD & (eqD - 1u)) != 0 || nextD || (hc >> 20) - (mD >> 20) > 18u;
  const int kC = (int)((0x6431u >> (4 * (__ffs(eqC) - 1))) & 15u);
  const int kD = (int)((0x7520u >> (4 * (__ffs(eqD) - 1))) & 15u);
  // slopes in FP32 from the high words (meaningful only when both minima
  // are within 18 binades of h_c, which the checks below require)
  const float fc = __uint_as_float((hc - (896u << 20)) << 3);
  const float sC = __fsub_rn(fc, __uint_as_float((mC - (896u << 20)) << 3));
  const float sD = __fmul_rn(__fsub_rn(fc, __uint_as_float((mD - (896u << 20)) << 3)), 0.70710677f);
  const float tol = __fmul_rn(__fadd_rn(fc, fmaxf(sC, sD)), 1.52587890625e-05f);  // 2^-16
  const bool cWins = __fsub_rn(sC, sD) > tol, dWins = __fsub_rn(sD, sC) > tol;
  // non-negative, finite, h_c (and anything within 18 binades below it) in
  // the float exponent range, and no neighbour group sharing h_c's high word
  const bool undecided = worst >= 0x7FF00000u || hc < (915u << 20) || hc >= (1151u << 20) ||
                         mC == hc || mD == hc || (hasC && badC) || (hasD && badD) ||
                         (hasC && hasD && !cWins && !dWins);
  const int code = !hasC ? (hasD ? kD : kSink) : (!hasD ? kC : (cWins ? kC : kD));
  return undecided ? -1 : code;
}

// receiver_code_hi_words for nine high words of finite non-negative values
// (the caller checks that for a whole strip at a time), given each group's
// smallest (mC, mD) and second smallest (rC, rD, counting repeats) high word:
// the minimum is unique and no member holds the next high word exactly when
// the second smallest is at least two above it.  The same result as
// receiver_code_hi_words for such values.
__device__ __forceinline__ int receiver_code_hi_nn(const unsigned hc, const unsigned* x,
                                                   unsigned mC, unsigned rC, unsigned mD,
                                                   unsigned rD) {
  const bool hasC = mC < hc, hasD = mD < hc;
  const bool badC = rC < mC + 2u || (hc >> 20) - (mC >> 20) > 18u;
  const bool badD = rD < mD + 2u || (hc >> 20) - (mD >> 20) > 18u;
  const int kC = x[1] == mC ? 1 : (x[3] == mC ? 3 : (x[4] == mC ? 4 : 6));
  const int kD = x[0] == mD ? 0 : (x[2] == mD ? 2 : (x[5] == mD ? 5 : 7));
  // slopes in FP32 from the high words, as in receiver_code_hi_words
  const float fc = __uint_as_float((hc - (896u << 20)) << 3);
  const float sC = __fsub_rn(fc, __uint_as_float((mC - (896u << 20)) << 3));
  const float sD = __fmul_rn(__fsub_rn(fc, __uint_as_float((mD - (896u << 20)) << 3)), 0.70710677f);
  const float tol = __fmul_rn(__fadd_rn(fc, fmaxf(sC, sD)), 1.52587890625e-05f);  // 2^-16
  const bool cWins = __fsub_rn(sC, sD) > tol, dWins = __fsub_rn(sD, sC) > tol;
  const bool undecided = hc < (915u << 20) || hc >= (1151u << 20) || mC == hc || mD == hc ||
                         (hasC && badC) || (hasD && badD) || (hasC && hasD && !cWins && !dWins);
  const bool pickC = hasC && (!hasD || cWins);
  const int code = pickC ? kC : (hasD ? kD : kSink);
  return undecided ? -1 : code;
}

__device__ __forceinline__ int receiver_code_hi(const double hcd, const double* v) {
  unsigned x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (unsigned)__double2hiint(v[k]);
  return receiver_code_hi_words((unsigned)__double2hiint(hcd), x);
}

// The group minima by bit patterns and the winners' slopes in FP64 (see
// above), without the high-word first try.
template <typename HT>
__device__ __forceinline__ int receiver_code_exact(const HT hcv, const HT* v) {
  using B = Bits<HT>;
  using U = typename B::U;
  const U bc = B::of(hcv);
  U mC = bc, mD = bc, rC = bc, rD = bc;  // group minima and runners-up below hc
  int kC = kSink, kD = kSink;
  U worst = bc;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const U x = B::of(v[k]);
    worst = x > worst ? x : worst;
    if (nbr_diag(k)) {
      if (x < mD) { rD = mD; mD = x; kD = k; }
      else if (x > mD && x < rD) rD = x;
    } else {
      if (x < mC) { rC = mC; mC = x; kC = k; }
      else if (x > mC && x < rC) rC = x;
    }
  }
  if (worst < B::kInf && no_rounding_merge<HT>(mC, rC, bc) &&
      no_rounding_merge<HT>(mD, rD, bc)) {
    if (kC == kSink && kD == kSink) return kSink;
    if (kD == kSink) return kC;
    if (kC == kSink) return kD;
    if constexpr (sizeof(HT) == 4) {
      // FP32 elevations: the FP32 slopes are within 4*2^-24 (relative) of the
      // FP64 ones, so they decide whenever they differ by more than 2^-18;
      // only near-ties (and tiny slopes) are compared in FP64.
      const float sCf = __fsub_rn(hcv, v[kC]);
      const float sDf = __fmul_rn(__fsub_rn(hcv, v[kD]), 0.70710677f);
      if (fminf(sCf, sDf) > 1e-30f) {
        if (sCf > __fmul_rn(sDf, 1.000003814697265625f)) return kC;
        if (sDf > __fmul_rn(sCf, 1.000003814697265625f)) return kD;
      }
    }
    const double hc = (double)hcv;
    const double sD = __dmul_rn(__dsub_rn(hc, (double)v[kD]), kInvSqrt2);
    const double sC = __dsub_rn(hc, (double)v[kC]);
    // both slopes are positive: compare their bit patterns
    const long long bC = __double_as_longlong(sC), bD = __double_as_longlong(sD);
    if (bC > bD) return kC;
    if (bD > bC) return kD;
    return min(kC, kD);
  }
  return receiver_code_slow((double)hcv, (double)v[0], (double)v[1], (double)v[2],
                            (double)v[3], (double)v[4], (double)v[5], (double)v[6],
                            (double)v[7]);
}

template <typename HT>
__device__ __forceinline__ int receiver_code_vals(const HT hcv, const HT* v) {
  if constexpr (sizeof(HT) == 8) {
    const int k = receiver_code_hi(hcv, v);
    if (k >= 0) return k;
  }
  return receiver_code_exact(hcv, v);
}

// Alg 1 for FP32 elevations: the same result as receiver_code<float>, with
// the group minima taken by float min/max (all nine values non-negative and
// finite, so min is exact and equality picks the lowest k).  The runner-up
// check is needed only when a minimum is 0 or more than 27 binades below h_c
// (otherwise distinct floats are always more than 4 FP64 ulps of h_c apart).
__device__ __forceinline__ bool f32_group_safe(const float* v, const int* ks, float m, float hc) {
  using B = Bits<float>;
  const unsigned bm = B::of(m), bc = B::of(hc);
  if (bm != 0 && (int)(bc >> 23) - max((int)(bm >> 23), 1) <= 27) return true;
  unsigned r = bc;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned x = B::of(v[ks[i]]);
    if (x > bm && x < r) r = x;
  }
  return no_rounding_merge<float>(bm, r, bc);
}

// The common case of receiver_code_f32_vals without branches: returns the
// code when every condition of its fast path holds (finite non-negative
// values, group minima nonzero and within 27 binades of h_c, FP32 slopes
// apart by more than 2^-18), else -1.
__device__ __forceinline__ int receiver_f32_fast(const float hc, const float* v) {
  const unsigned bc = __float_as_uint(hc);
  unsigned worst = bc;
#pragma unroll
  for (int k = 0; k < 8; ++k) worst = max(worst, __float_as_uint(v[k]));
  const float mC = fminf(fminf(v[1], v[3]), fminf(v[4], v[6]));
  const float mD = fminf(fminf(v[0], v[2]), fminf(v[5], v[7]));
  const bool hasC = mC < hc, hasD = mD < hc;
  const int kC = v[1] == mC ? 1 : (v[3] == mC ? 3 : (v[4] == mC ? 4 : 6));
  const int kD = v[0] == mD ? 0 : (v[2] == mD ? 2 : (v[5] == mD ? 5 : 7));
  // a minimum m qualifies if m >= max(h_c 2^-27, 2^-126): then m is normal
  // and at most 27 binades below h_c (h_c 2^-27 is exact whenever it is at
  // least 2^-126), a subset of the exponent test of f32_group_safe
  const float thr = fmaxf(__fmul_rn(hc, 0x1p-27f), 0x1p-126f);
  const bool okC = mC >= thr, okD = mD >= thr;
  const float sC = __fsub_rn(hc, mC);
  const float sD = __fmul_rn(__fsub_rn(hc, mD), 0.70710677f);
  const bool cWins = sC > __fmul_rn(sD, 1.000003814697265625f);
  const bool dWins = sD > __fmul_rn(sC, 1.000003814697265625f);
  const bool both = hasC && hasD;
  const bool undecided = worst >= Bits<float>::kInf || (hasC && !okC) || (hasD && !okD) ||
                         (both && (!(fminf(sC, sD) > 1e-30f) || (!cWins && !dWins)));
  const int code = !hasC ? (hasD ? kD : kSink) : (!hasD ? kC : (cWins ? kC : kD));
  return undecided ? -1 : code;
}

// receiver_f32_fast for nine values that are all finite and non-negative
// (the caller checks that separately, for a whole strip at a time), given
// the bit patterns bC, bD of the cardinal and diagonal minima (for such
// values bit patterns order as the values do).  Returns the same as
// receiver_f32_fast for such values, or -1 (undecided) in more cases: a
// minimum must be at least max(h_c 2^-27, 2^-76), which keeps both FP32
// slopes of a two-group decision above 2^-99 (so above the 1e-30 floor of
// receiver_f32_fast without testing it).
__device__ __forceinline__ int receiver_f32_fast_nn(const float hc, const float* v, unsigned bC,
                                                    unsigned bD) {
  const unsigned bc = __float_as_uint(hc);
  const float mC = __uint_as_float(bC), mD = __uint_as_float(bD);
  const bool hasC = bC < bc, hasD = bD < bc;
  const int kC = v[1] == mC ? 1 : (v[3] == mC ? 3 : (v[4] == mC ? 4 : 6));
  const int kD = v[0] == mD ? 0 : (v[2] == mD ? 2 : (v[5] == mD ? 5 : 7));
  const float thr = fmaxf(__fmul_rn(hc, 0x1p-27f), 0x1p-76f);
  const bool okC = mC >= thr, okD = mD >= thr;
  const float sC = __fsub_rn(hc, mC);
  const float sD = __fmul_rn(__fsub_rn(hc, mD), 0.70710677f);
  const bool cWins = sC > __fmul_rn(sD, 1.000003814697265625f);
  const bool dWins = sD > __fmul_rn(sC, 1.000003814697265625f);
  const bool undecided =
      (hasC && !okC) || (hasD && !okD) || (hasC && hasD && !cWins && !dWins);
  const bool pickC = hasC && (!hasD || cWins);
  const int code = pickC ? kC : (hasD ? kD : kSink);
  return undecided ? -1 : code;
}

// st: where a non-finite value among the nine is reported (kErrInval); the
// check runs only on the path that such values take (bit patterns at or
// above that of +inf, which negative values share).
__device__ __forceinline__ int receiver_code_f32_vals(const float hc, const float* v,
                                                      DevState* st = nullptr) {
  {
    const int k = receiver_f32_fast(hc, v);
    if (k >= 0) return k;
  }
  unsigned worst = Bits<float>::of(hc);
#pragma unroll
  for (int k = 0; k < 8; ++k) worst = max(worst, Bits<float>::of(v[k]));
  if (worst >= Bits<float>::kInf && st) {
    bool fin = isfinite(hc);
#pragma unroll
    for (int k = 0; k < 8; ++k) fin = fin && isfinite(v[k]);
    if (!fin) set_error(st, kErrInval);
  }
  if (worst < Bits<float>::kInf) {
    const float mC = fminf(fminf(v[1], v[3]), fminf(v[4], v[6]));
    const float mD = fminf(fminf(v[0], v[2]), fminf(v[5], v[7]));
    const bool hasC = mC < hc, hasD = mD < hc;
    if (!hasC && !hasD) return kSink;
    const int kC = v[1] == mC ? 1 : (v[3] == mC ? 3 : (v[4] == mC ? 4 : 6));
    const int kD = v[0] == mD ? 0 : (v[2] == mD ? 2 : (v[5] == mD ? 5 : 7));
    const int cks[4] = {1, 3, 4, 6}, dks[4] = {0, 2, 5, 7};
    if ((!hasC || f32_group_safe(v, cks, mC, hc)) && (!hasD || f32_group_safe(v, dks, mD, hc))) {
      if (!hasD) return kC;
      if (!hasC) return kD;
      const float sCf = __fsub_rn(hc, mC);
      const float sDf = __fmul_rn(__fsub_rn(hc, mD), 0.70710677f);
      if (fminf(sCf, sDf) > 1e-30f) {
        if (sCf > __fmul_rn(sDf, 1.000003814697265625f)) return kC;
        if (sDf > __fmul_rn(sCf, 1.000003814697265625f)) return kD;
      }
      const double hcd = (double)hc;
      const double sC = __dsub_rn(hcd, (double)mC);
      const double sD = __dmul_rn(__dsub_rn(hcd, (double)mD), kInvSqrt2);
      const long long bC = __double_as_longlong(sC), bD = __double_as_longlong(sD);
      if (bC > bD) return kC;
      if (bD > bC) return kD;
      return min(kC, kD);
    }
  }
  return receiver_code_slow((double)hc, (double)v[0], (double)v[1], (double)v[2], (double)v[3],
                            (double)v[4], (double)v[5], (double)v[6], (double)v[7]);
}

// Alg 1 for an interior cell of elevation hc with neighbour elevations
// v[0..7] (k order).
template <typename HT>
__device__ __forceinline__ int receiver_from(const HT hc, const HT* v, DevState* st = nullptr) {
  if constexpr (sizeof(HT) == 4) {
    return receiver_code_f32_vals(hc, v, st);
  } else {
    return receiver_code_vals(hc, v);
  }
}

// ---- Alg 5 + Alg 6 -------------------------------------------------------------

template <typename HT, typename CT>
__device__ __forceinline__ double uplift_dt(const StepArgs<HT, CT>& a, int c) {
  return a.Uf ? __dmul_rn(a.Uf[c], a.dt) : a.Udt;
}

template <typename HT, typename CT>
__device__ __forceinline__ float uplift_dt_f(const StepArgs<HT, CT>& a, int c) {
  return a.Uf ? (float)__dmul_rn(a.Uf[c], a.dt) : a.Udt_f;
}

// Alg 5 for a cell without receiver: pits are uplifted, the perimeter is not.
template <typename HT, typename CT>
__device__ __forceinline__ void uplift_sink(const StepArgs<HT, CT>& a, int c) {
  if (a.code[c] != kSink) return;
  if constexpr (sizeof(HT) == 8) {
    a.h[c] = __dadd_rn(a.h[c], uplift_dt(a, c));
  } else {
    a.h[c] = __fadd_rn(a.h[c], uplift_dt_f(a, c));
  }
}

// The n = 1 implicit update for one cell of level >= 1, given its receiver
// code k, count, own elevation hcur and the receiver's updated elevation hr.
// The closed form h = (h0 + F*hr)/(1+F), h0 = h + dt*U, is evaluated in the
// algebraically identical increment form h = h0 - g*(h0 - hr) with
// g = F/(1+F) taken from a table (computed in FP64 by division for every
// count below kTableN): one subtraction and one fused multiply-add per cell
// instead of a division, which GB300 runs about seven times slower than an
// FMA in FP64.  The results differ from the closed form by a few units in the
// last place.  FP32 elevations use the same form with g rounded once to float.
// g = F/(1+F) for a count beyond the tables, the same operations as the
// tables (FP64 division; for FP32 contexts rounded to float by the caller).
template <typename HT, typename CT>
__device__ __forceinline__ double big_count_g(const StepArgs<HT, CT>& a, CT count, bool diag) {
  if constexpr (sizeof(HT) == 8) {
    const double A = __dmul_rn((double)count, a.area_scale);
    const double F = __ddiv_rn(__dmul_rn(a.Kdt, pow(A, a.m)), diag ? a.dxd : a.dx);
    return __ddiv_rn(F, __dadd_rn(1.0, F));
  } else {
    const double A = (double)count * a.area_scale;
    const double F = a.Kdt * pow(A, a.m) / (diag ? a.dxd : a.dx);
    return F / (1.0 + F);
  }
}

// The erosion factor g = F/(1+F) of a cell (double for FP64 elevations,
// float for FP32).  gbig: when not null, big_count_g of every cell whose
// count is beyond the tables, computed ahead of the level sweep
// (phase_global_erode).
template <typename HT, typename CT>
__device__ __forceinline__ HT erode_factor(const StepArgs<HT, CT>& a, int c, int k, CT count,
                                           const double* gbig) {
  const bool diag = nbr_diag(k);
  if constexpr (sizeof(HT) == 8) {
    if (count < (CT)kTableN) return a.Ftab[(diag ? kTableN : 0) + (int)count].y;
    return gbig ? gbig[c] : big_count_g(a, count, diag);
  } else {
    if (count < (CT)kTableN) return a.gtab[(diag ? kTableN : 0) + (int)count];
    return (float)(gbig ? gbig[c] : big_count_g(a, count, diag));
  }
}

// The increment form with a given factor g.
template <typename HT, typename CT>
__device__ __forceinline__ HT erode_apply(const StepArgs<HT, CT>& a, int c, HT g, HT hcur,
                                          HT hr) {
  if constexpr (sizeof(HT) == 8) {
    const double h0 = __dadd_rn(hcur, uplift_dt(a, c));
    return __fma_rn(-g, __dsub_rn(h0, hr), h0);
  } else {
    const float h0 = __fadd_rn(hcur, uplift_dt_f(a, c));
    return __fmaf_rn(-g, __fsub_rn(h0, hr), h0);
  }
}

template <typename HT, typename CT>
__device__ __forceinline__ HT erode_value(const StepArgs<HT, CT>& a, int c, int k, CT count,
                                          HT hcur, HT hr) {
  return erode_apply(a, c, erode_factor(a, c, k, count, (const double*)nullptr), hcur, hr);
}

// Alg 6 for a general slope exponent n (Eq. 1 with S^n): Newton-Raphson on
// f(h) = h - h0 + F*(h - hr)^n from h = h0 = h + dt*U, F = K*dt*A^m / d^n,
// stopped once an update moves h by at most eps or after newton_iters
// updates.  FP64 for either elevation type.  For n >= 1, f is convex and
// increasing above hr, so the iterates fall monotonically to the root and
// stay above hr.  A cell whose h0 is not above hr keeps h0: the power of a
// non-positive slope is undefined for non-integer n.  The step kernel has an
// instantiation of its own for it (lem_step_kernel<HT, CT, true>), so the
// n = 1 kernel is compiled without it.
// The Newton-Raphson iteration of Alg 6 for one cell: the root of
// h - h0 + F*(h - hr)^n from h = h0; h0 itself if it is not above hr.
static __device__ __noinline__ double newton_solve(double h0, double hr, double F, double n,
                                                   double eps,
                                            int iters) {
  if (!(h0 - hr > 0.0)) return h0;
  double hn = h0, hp = h0;
  for (int it = 0; it < iters; ++it) {
    const double x = hn - hr;
    // x^(n-1), as 2^((n-1) log2 x): two FP64 library calls instead of the
    // costlier general power, within a few units in the last place of it
    const double p = (n == 2.0) ? x : exp2((n - 1.0) * log2(x));
    const double f = (hn - h0) + F * (p * x);
    const double fp = 1.0 + F * n * p;
    hn = hn - f / fp;
    const double d = hn - hp;
    hp = hn;
    if (!(fabs(d) > eps)) break;
  }
  return hn;
}

template <typename HT, typename CT>
__device__ __forceinline__ HT erode_newton(const StepArgs<HT, CT>& a, int c, int k, CT count,
                                           HT hcur, HT hrecv) {
  const double h0 = (double)hcur + uplift_dt(a, c);
  // F = K*dt*A^m / d^n: for tabulated counts the n = 1 factor times d^(1-n)
  const bool diag = nbr_diag(k);
  double F;
  if (count < (CT)kTableN) {
    F = a.Ftab[(diag ? kTableN : 0) + (int)count].x * (diag ? a.dfacd : a.dfac);
  } else {
    const double A = (double)count * a.area_scale;
    F = a.Kdt * pow(A, a.m) / (diag ? a.dxdn : a.dxn);
  }
  return (HT)newton_solve(h0, (double)hrecv, F, a.nexp, a.neps, a.newton_iters);
}

// Erode up to kItems cells (entries < 0 are skipped) with all loads issued
// before the arithmetic.
template <bool kNewton, typename HT, typename CT>
__device__ __forceinline__ void erode_items(const StepArgs<HT, CT>& a, const int* cs,
                                            const double* gbig) {
  int ks[kItems];
  CT ns[kItems];
  HT hc[kItems], hr[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if (cs[i] >= 0) {
      ks[i] = a.code[cs[i]];
      ns[i] = a.cnt[cs[i]];
      hc[i] = a.h[cs[i]];
    }
  }
#pragma unroll
  for (int i = 0; i < kItems; ++i)
    if (cs[i] >= 0) hr[i] = a.h[cs[i] + nbr_off(ks[i], a.nx)];
  if constexpr (kNewton) {
    for (int i = 0; i < kItems; ++i)
      if (cs[i] >= 0 && in_bounds(a.st, cs[i], a.N))
        a.h[cs[i]] = erode_newton(a, cs[i], ks[i], ns[i], hc[i], hr[i]);
  } else {
#pragma unroll
    for (int i = 0; i < kItems; ++i)
      if (cs[i] >= 0 && in_bounds(a.st, cs[i], a.N))
        a.h[cs[i]] = erode_apply(a, cs[i], erode_factor(a, cs[i], ks[i], ns[i], gbig), hc[i],
                                 hr[i]);
  }
}

// ---- Alg 4 ------------------------------------------------------------------------

template <typename CT>
__device__ __forceinline__ CT donor_sum(const CT* __restrict__ cnt, int c, int msk, int nx) {
  CT s = 1;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if ((msk >> k) & 1) s += cnt[c + nbr_off(k, nx)];
  return s;
}

template <typename HT, typename CT>
__device__ __forceinline__ void accumulate_items(const StepArgs<HT, CT>& a, const int* cs) {
  int ms[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) ms[i] = (cs[i] >= 0) ? a.mask[cs[i]] : 0;
  CT s[kItems];
#pragma unroll
  for (int i = 0; i < kItems; ++i) s[i] = donor_sum(a.cnt, cs[i], ms[i], a.nx);
#pragma unroll
  for (int i = 0; i < kItems; ++i)
    if (cs[i] >= 0 && in_bounds(a.st, cs[i], a.N)) a.cnt[cs[i]] = s[i];
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

// Sum of a per-block value over blocks [0, b) and over all blocks.
template <int BD>
__device__ __forceinline__ void block_prefix_of_partials(const int* partial, int G, int b,
                                                         int* prefix, int* total,
                                                         long long* s_sum) {
  long long p = 0, s = 0;
  for (int i = threadIdx.x; i < G; i += BD) {
    const int v = partial[i];
    s += v;
    if (i < b) p += v;
  }
  *prefix = (int)block_sum<BD>(p, s_sum);
  *total = (int)block_sum<BD>(s, s_sum);
}

struct Shared {
  int scan[kWarps];
  long long sum[kWarps];
  int wcount[kWarps];
  int chunk[kPItems * kWarps];  // per (slot, warp) donor totals, then offsets
  int chunk_total;
  int n_ovf, n0;                // block tier: overflowed work items, roots
  int off[8];                   // address offset of neighbour k
  int ovf_tiles[kOvfCap];       // overflowed work items (tile_item packing)
};
static_assert(kPItems * kWarps == 8 * 32, "one warp scans the chunk totals 8 per lane");

// ---- phase: Alg 1 receivers, Alg 2 donor masks, level 0 of Alg 3 ---------------

// Block b's chunk of cells and warp w's sub-chunk of it; both start at
// multiples of 4 cells (128 per warp round).
__device__ __forceinline__ void warp_range(int N, int G, int b, int w, int* w0, int* w1) {
  const int chunk = ((N + G - 1) / G + 127) & ~127;
  const int c0 = min(N, b * chunk), c1 = min(N, c0 + chunk);
  const int wchunk = ((c1 - c0 + kWarps - 1) / kWarps + 127) & ~127;
  *w0 = min(c1, c0 + w * wchunk);
  *w1 = min(c1, *w0 + wchunk);
}

// Algs 1-2 for the tiered step.  A warp owns a strip of kStripOut columns
// and strip_rows() rows at a time.  It first stages the elevations the strip
// needs (two rows and columns of halo on each side) into its slice of shared
// memory with asynchronous copies, all in flight at once; then lane l walks
// down column x0 - 1 + l (lanes 0 and 31 are halo columns) with a 3x3 window
// in registers.  Receiver codes are computed for the strip's rows and one
// halo row above and below, so the donor mask of each owned cell (Alg 2)
// follows from the codes of its 3x3 neighbourhood, exchanged by shuffles.
// Cells outside the grid count as code 0xFF (no receiver anywhere), which
// leaves the perimeter cells' masks exact.
constexpr int kStripOut = 30;                // owned columns per strip (lanes 1..30)
// owned rows per strip, at most: 32 with FP32 elevations, 16 with FP64
// (whose staged strip must also fit a warp's slice of shared memory).  A
// pass takes 16-row strips when the taller ones would leave fewer than two
// per warp (pick_strip_rows).
template <typename HT>
__host__ __device__ constexpr int strip_rows() {
  return sizeof(HT) == 4 ? 32 : 16;
}
// staged rows at most: two of halo on each side
template <typename HT>
__host__ __device__ constexpr int stage_rows() {
  return strip_rows<HT>() + 4;
}
template <typename HT>
__host__ __device__ __forceinline__ int pick_strip_rows(int nx, int ny, int warps) {
  constexpr int R = strip_rows<HT>();
  const long long tall = (long long)((nx + kStripOut - 1) / kStripOut) * ((ny + R - 1) / R);
  return (R > 16 && tall < 2LL * warps) ? 16 : R;
}
constexpr int kStageCols = 36;               // staged columns (16-byte aligned start)

template <typename HT>
__device__ __forceinline__ void cp_async_elem(HT* dst, const HT* src, bool in) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src),
               "n"((int)sizeof(HT)), "r"(in ? (int)sizeof(HT) : 0)
               : "memory");
}

// Stage rows [yb, yb + rows) x columns [xb, xb + kStageCols) of h into
// S (row-major); positions outside the grid are zero-filled.
template <typename HT>
__device__ __forceinline__ void stage_strip(const HT* h, int nx, int ny, int xb, int yb, int rows,
                                            HT* S, int lane) {
  for (int i = lane; i < rows * kStageCols; i += 32) {
    const int r = i / kStageCols, col = i - r * kStageCols;
    const int x = xb + col, y = yb + r;
    const bool in = x >= 0 && x < nx && y >= 0 && y < ny;
    cp_async_elem(S + i, in ? h + ((size_t)y * nx + x) : h, in);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
}

// ---- TMA and mbarrier primitives (inline PTX, sm_90+) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Order this thread's earlier generic accesses to shared memory before
// later asynchronous-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 2-D tiled TMA load of the box at element coordinates (x, y) into dst,
// completing on bar.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Hint the TMA unit to bring the box at (x, y) into L2 (no shared memory
// involved, nothing to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const void* tmap, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(tmap),
               "r"(x), "r"(y)
               : "memory");
}

// Wait for phase `parity` of bar, bounded by the context's wait limit.
// Returns false (with kErrTimeout recorded) if the limit ran out or another
// block recorded an error.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, DevState* st) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  unsigned it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++it & 255u) == 0) {
      if (ld_volatile(&st->err) != 0) return false;
      if (global_ns() - t0 > st->wait_limit_ns) {
        set_error(st, kErrTimeout);
        return false;
      }
    }
  }
  return true;
}

// A cell's receiver code as a one-hot byte: bit d set when it drains to its
// neighbour d, zero without receiver (codes 8, 9) or outside the grid (0xFF).
__device__ __forceinline__ unsigned pointer_bits(int cd) { return cd < 8 ? 1u << cd : 0u; }

// Donor mask from packed pointer bytes (byte 0 = row above, 1 = own row, 2 =
// row below) of the left lane (pl), this lane (pw) and the right lane (pr).
// Neighbour k drains into the cell iff its byte has bit 7-k: NW bit 7, N 6,
// NE 5 above; W 4, E 3 beside; SW 2, S 1, SE 0 below.  Those eight bits are
// disjoint, so they fold into one byte t with bit 7-k for neighbour k, and
// the mask (bit k for neighbour k) is t bit-reversed.
__device__ __forceinline__ int mask_from_pointers(unsigned pl, unsigned pw, unsigned pr) {
  const unsigned v = (pl & 0x041080u) | (pw & 0x020040u) | (pr & 0x010820u);
  const unsigned t = (v | (v >> 8) | (v >> 16)) & 0xFFu;
  return (int)(__brev(t) >> 24);
}

// Algs 1-2 on one staged strip: S holds rows y0-2 .. y0+rows+1 and
// columns xb .. xb+kStageCols-1 of the elevations (zero outside the grid).
// Lane l walks column x0 - 1 + l down the strip with a 3 x 3 window in
// registers and writes the codes and masks of the owned cells (lanes 1 ..
// kStripOut, rows y0 .. y0+rows-1, inside the grid).  With frozen
// receivers the codes are read instead of computed.
// codes_strip for FP64 elevations: the register window holds only the high
// words of the values (receiver_code_hi_words decides from them alone); a
// cell it leaves undecided reloads its nine doubles from the staged strip
// for the exact comparison.
template <bool B>
struct RowKind {
  static constexpr bool general = B;
};
// A compile-time flag passed as a value (for generic lambdas).
template <bool B>
struct Flag {
  static constexpr bool value = B;
};
// Smallest and second smallest (counting repeats) of two sorted pairs.
struct Low2 {
  unsigned lo, hi;
};
__device__ __forceinline__ Low2 low2(unsigned a, unsigned b) { return Low2{min(a, b), max(a, b)}; }
__device__ __forceinline__ Low2 low2(Low2 p, Low2 q) {
  return Low2{min(p.lo, q.lo), __vimin3_u32(max(p.lo, q.lo), p.hi, q.hi)};
}
__device__ __forceinline__ void codes_strip_f64(const double* S, uint8_t* code, uint8_t* mask,
                                                int nx, int ny, int x, int y0, int y1, bool xin,
                                                bool xperim, bool own, int sc, DevState* st) {
  const int yb = y0 - 2;
  const long long N = (long long)nx * ny;
  // high word of staged element (row r, column col)
  auto hw = [&](int r, int col) -> unsigned {
    return reinterpret_cast<const unsigned*>(S + r * kStageCols + col)[1];
  };
  // the exact comparison for a cell the high words leave undecided, its
  // nine doubles reloaded from the staged strip (r: staged row below it)
  auto exact = [&](int r) -> int {
    const double* up = S + (r - 2) * kStageCols + sc;
    const double* md = up + kStageCols;
    const double* dn = md + kStageCols;
    const double v[8] = {up[-1], up[0], up[1], md[-1], md[1], dn[-1], dn[0], dn[1]};
    if (st) {
      // non-finite elevations are rejected (reported as kErrInval)
      bool fin = isfinite(md[0]);
#pragma unroll
      for (int k = 0; k < 8; ++k) fin = fin && isfinite(v[k]);
      if (!fin) set_error(st, kErrInval);
    }
    return receiver_code_vals(md[0], v);
  };
  // one pass over the strip: high-word decisions (a running maximum of every
  // high word read is returned), or with kExact every interior cell exact
  auto pass = [&](auto exact_kind) -> unsigned {
    constexpr bool kExact = decltype(exact_kind)::value;
    unsigned ul = hw(0, sc - 1), uc = hw(0, sc), ur = hw(0, sc + 1);
    unsigned ml = hw(1, sc - 1), mc = hw(1, sc), mr = hw(1, sc + 1);
    unsigned worst = max(__vimax3_u32(ul, uc, ur), __vimax3_u32(ml, mc, mr));
    long long at = (long long)(y0 - 1) * nx + x;
    unsigned pw = 0;
    // two rows per iteration (y and y + 1): their receiver decisions are
    // independent, so the scheduler can interleave them; iterations whose
    // rows are both owned interior rows skip the per-row tests
    auto rows = [&](auto kind, int y) {
      constexpr bool general = decltype(kind)::general;
      const bool two = !general || y + 1 <= y1;  // the same for the whole warp
      const int r = y + 1 - yb;                  // staged row below row y
      const int r2 = two ? r + 1 : r;
      const unsigned dl = hw(r, sc - 1), dc = hw(r, sc), dr = hw(r, sc + 1);
      const unsigned el = hw(r2, sc - 1), ec = hw(r2, sc), er = hw(r2, sc + 1);
      worst = __vimax3_u32(worst, __vimax3_u32(dl, dc, dr), __vimax3_u32(el, ec, er));
      bool in0 = xin, in1 = xin, edge0 = xperim, edge1 = xperim;
      if constexpr (general) {
        in0 = xin && y >= 0 && y < ny;
        in1 = two && xin && y + 1 < ny;  // y + 1 >= 0 always
        edge0 = xperim || y == 0 || y == ny - 1;
        edge1 = xperim || y + 1 == 0 || y + 1 == ny - 1;
      }
      int c0, c1;
      if constexpr (kExact) {
        c0 = !in0 ? 0xFF : (edge0 ? kEdge : exact(r));
        c1 = !in1 ? 0xFF : (edge1 ? kEdge : exact(r2));
      } else {
        // group minima and runners-up: W-E of row y is diagonal to row
        // y + 1, and SW-SE of row y is cardinal to it
        const Low2 pWE = low2(ml, mr), pS = low2(dl, dr);
        const Low2 gC0 = low2(pWE, low2(uc, dc)), gD0 = low2(low2(ul, ur), pS);
        const Low2 gC1 = low2(pS, low2(mc, ec)), gD1 = low2(pWE, low2(el, er));
        const unsigned xs0[8] = {ul, uc, ur, ml, mr, dl, dc, dr};
        const unsigned xs1[8] = {ml, mc, mr, dl, dr, el, ec, er};
        c0 = receiver_code_hi_nn(mc, xs0, gC0.lo, gC0.hi, gD0.lo, gD0.hi);
        c1 = receiver_code_hi_nn(dc, xs1, gC1.lo, gC1.hi, gD1.lo, gD1.hi);
        c0 = !in0 ? 0xFF : (edge0 ? kEdge : c0);
        c1 = !in1 ? 0xFF : (edge1 ? kEdge : c1);
        // cells the high words leave open take the exact comparison, behind
        // a warp-uniform branch so that the other cells do not execute it
        if (__builtin_expect(__any_sync(0xffffffffu, c0 < 0 || c1 < 0), 0)) {
          if (c0 < 0) c0 = exact(r);
          if (c1 < 0) c1 = exact(r2);
        }
      }
      if constexpr (general) {
        if (own && in0 && y >= y0 && y < y1 && in_bounds(st, at, N)) code[at] = (uint8_t)c0;
        if (own && in1 && y + 1 < y1 && in_bounds(st, at + nx, N)) code[at + nx] = (uint8_t)c1;
      } else if (own) {
        if (in_bounds(st, at, N)) code[at] = (uint8_t)c0;
        if (in_bounds(st, at + nx, N)) code[at + nx] = (uint8_t)c1;
      }
      pw = ((pw >> 8) & 0xFFFFu) | (pointer_bits(c0) << 16);
      unsigned pl = __shfl_up_sync(0xffffffffu, pw, 1);
      unsigned pr = __shfl_down_sync(0xffffffffu, pw, 1);
      const int m0 = mask_from_pointers(pl, pw, pr);
      if (own && (!general || (y > y0 && y <= y1)) && in_bounds(st, at - nx, N))
        mask[at - nx] = (uint8_t)m0;
      if (two) {
        pw = ((pw >> 8) & 0xFFFFu) | (pointer_bits(c1) << 16);
        pl = __shfl_up_sync(0xffffffffu, pw, 1);
        pr = __shfl_down_sync(0xffffffffu, pw, 1);
        const int m1 = mask_from_pointers(pl, pw, pr);
        if (own && (!general || y + 1 > y0) && in_bounds(st, at, N)) mask[at] = (uint8_t)m1;
      }
      ul = dl; uc = dc; ur = dr;
      ml = el; mc = ec; mr = er;
    };
    int y = y0 - 1;
    rows(RowKind<true>{}, y);
    y += 2;
    at += 2 * (long long)nx;
    const int ylim = min(y1 - 1, ny - 2);
    for (; y + 1 <= ylim; y += 2, at += 2 * (long long)nx) rows(RowKind<false>{}, y);
    for (; y <= y1; y += 2, at += 2 * (long long)nx) rows(RowKind<true>{}, y);
    return worst;
  };
  // a strip that held a negative or non-finite value (a high word at or
  // above that of +inf) is redone with every interior cell exact, which
  // also reports non-finite values
  if (__any_sync(0xffffffffu, pass(Flag<false>{}) >= 0x7FF00000u)) pass(Flag<true>{});
}

// codes_strip for FP32 elevations: two rows per iteration, as the FP64 form
// (their decisions are independent, so the scheduler can interleave them);
// the fast FP32 decision, and the exact one for the cells it leaves open
// behind a warp-uniform branch (which also reports non-finite values).
// Iterations whose two rows are both owned and neither is a perimeter row
// (all but the first and the last one or two of a strip) run a form of the
// body without the per-row tests of the others.  The decisions assume
// finite non-negative values (receiver_f32_fast_nn); every staged value a
// lane reads goes into a running maximum of bit patterns, and a strip that
// held a negative or non-finite value returns false: the caller then redoes
// it with the per-cell checked form (which also reports non-finite values).
__device__ __forceinline__ bool codes_strip_f32(const float* S, uint8_t* code, uint8_t* mask,
                                                int nx, int ny, int x, int y0, int y1, bool xin,
                                                bool xperim, bool own, int sc, DevState* st) {
  const int yb = y0 - 2;
  auto el = [&](int r, int col) -> float { return S[r * kStageCols + col]; };
  auto bmax3 = [](float a, float b, float c) {
    return __vimax3_u32(__float_as_uint(a), __float_as_uint(b), __float_as_uint(c));
  };
  float ul = el(0, sc - 1), uc = el(0, sc), ur = el(0, sc + 1);
  float ml = el(1, sc - 1), mc = el(1, sc), mr = el(1, sc + 1);
  unsigned worst = max(bmax3(ul, uc, ur), bmax3(ml, mc, mr));
  long long at = (long long)(y0 - 1) * nx + x;
  const long long N = (long long)nx * ny;
  unsigned pw = 0;
  auto rows = [&](auto kind, int y) {
    constexpr bool general = decltype(kind)::general;
    const bool two = !general || y + 1 <= y1;  // the same for the whole warp
    const int r = y + 1 - yb;                  // staged row below row y
    const int r2 = two ? r + 1 : r;
    const float dl = el(r, sc - 1), dc = el(r, sc), dr = el(r, sc + 1);
    const float fl = el(r2, sc - 1), fc = el(r2, sc), fr = el(r2, sc + 1);
    const float v0[8] = {ul, uc, ur, ml, mr, dl, dc, dr};
    const float v1[8] = {ml, mc, mr, dl, dr, fl, fc, fr};
    worst = __vimax3_u32(worst, bmax3(dl, dc, dr), bmax3(fl, fc, fr));
    // group minima of both cells: W-E of row y is diagonal to row y + 1, and
    // SW-SE of row y is cardinal to it
    const unsigned p1 = min(__float_as_uint(ml), __float_as_uint(mr));
    const unsigned p2 = min(__float_as_uint(dl), __float_as_uint(dr));
    const unsigned bC0 = __vimin3_u32(__float_as_uint(uc), __float_as_uint(dc), p1);
    const unsigned bD0 = __vimin3_u32(__float_as_uint(ul), __float_as_uint(ur), p2);
    const unsigned bC1 = __vimin3_u32(__float_as_uint(mc), __float_as_uint(fc), p2);
    const unsigned bD1 = __vimin3_u32(__float_as_uint(fl), __float_as_uint(fr), p1);
    int c0 = receiver_f32_fast_nn(mc, v0, bC0, bD0);
    int c1 = receiver_f32_fast_nn(dc, v1, bC1, bD1);
    if constexpr (general) {
      const bool in0 = xin && y >= 0 && y < ny;
      const bool in1 = two && xin && y + 1 < ny;  // y + 1 >= 0 always
      c0 = !in0 ? 0xFF : ((xperim || y == 0 || y == ny - 1) ? kEdge : c0);
      c1 = !in1 ? 0xFF : ((xperim || y + 1 == 0 || y + 1 == ny - 1) ? kEdge : c1);
    } else {
      c0 = !xin ? 0xFF : (xperim ? kEdge : c0);
      c1 = !xin ? 0xFF : (xperim ? kEdge : c1);
    }
    if (__builtin_expect(__any_sync(0xffffffffu, c0 < 0 || c1 < 0), 0)) {
      if (c0 < 0) c0 = receiver_code_f32_vals(mc, v0, st);
      if (c1 < 0) c1 = receiver_code_f32_vals(dc, v1, st);
    }
    if constexpr (general) {
      const bool in0 = xin && y >= 0 && y < ny;
      const bool in1 = two && xin && y + 1 < ny;
      if (own && in0 && y >= y0 && y < y1 && in_bounds(st, at, N)) code[at] = (uint8_t)c0;
      if (own && in1 && y + 1 < y1 && in_bounds(st, at + nx, N)) code[at + nx] = (uint8_t)c1;
    } else if (own) {
      if (in_bounds(st, at, N)) code[at] = (uint8_t)c0;
      if (in_bounds(st, at + nx, N)) code[at + nx] = (uint8_t)c1;
    }
    pw = ((pw >> 8) & 0xFFFFu) | (pointer_bits(c0) << 16);
    unsigned pl = __shfl_up_sync(0xffffffffu, pw, 1);
    unsigned pr = __shfl_down_sync(0xffffffffu, pw, 1);
    const int m0 = mask_from_pointers(pl, pw, pr);
    if (own && (!general || (y > y0 && y <= y1)) && in_bounds(st, at - nx, N))
      mask[at - nx] = (uint8_t)m0;
    if (two) {
      pw = ((pw >> 8) & 0xFFFFu) | (pointer_bits(c1) << 16);
      pl = __shfl_up_sync(0xffffffffu, pw, 1);
      pr = __shfl_down_sync(0xffffffffu, pw, 1);
      const int m1 = mask_from_pointers(pl, pw, pr);
      if (own && (!general || y + 1 > y0) && in_bounds(st, at, N)) mask[at] = (uint8_t)m1;
    }
    ul = dl; uc = dc; ur = dr;
    ml = fl; mc = fc; mr = fr;
  };
  // rows y0 - 1 and y0 (row y0 - 1: codes for row y0's mask only)
  int y = y0 - 1;
  rows(RowKind<true>{}, y);
  y += 2;
  at += 2 * (long long)nx;
  // rows y, y + 1 both owned (y + 1 < y1) and in [1, ny - 2]: y >= y0 + 1 >= 1
  const int ylim = min(y1 - 1, ny - 2);
  for (; y + 1 <= ylim; y += 2, at += 2 * (long long)nx) rows(RowKind<false>{}, y);
  for (; y <= y1; y += 2, at += 2 * (long long)nx) rows(RowKind<true>{}, y);
  return !__any_sync(0xffffffffu, worst >= Bits<float>::kInf);
}

template <typename HT>
__device__ __forceinline__ void codes_strip(const HT* S, uint8_t* code, uint8_t* mask, int nx,
                                            int ny, int x0, int y0, int rows, int xb, bool frozen,
                                            int lane, DevState* st = nullptr) {
  const int x = x0 - 1 + lane;  // this lane's column
  const int y1 = min(ny, y0 + rows), yb = y0 - 2;
  const bool xin = x >= 0 && x < nx;
  const bool xperim = x == 0 || x == nx - 1;
  const bool own = lane >= 1 && lane <= kStripOut && xin;
  const int sc = x - xb;  // staged column of this lane's cell, 1..35
  if constexpr (sizeof(HT) == 8) {
    if (!frozen) {
      codes_strip_f64(reinterpret_cast<const double*>(S), code, mask, nx, ny, x, y0, y1, xin,
                      xperim, own, sc, st);
      return;
    }
  } else {
    // a strip holding a negative or non-finite value is redone below, cell by
    // cell with the checked decision
    if (!frozen && codes_strip_f32(reinterpret_cast<const float*>(S), code, mask, nx, ny, x, y0,
                                   y1, xin, xperim, own, sc, st))
      return;
  }
  HT ul = HT(0), uc = HT(0), ur = HT(0), ml = HT(0), mc = HT(0), mr = HT(0);
  if (!frozen) {
    ul = S[sc - 1];
    uc = S[sc];
    ur = S[sc + 1];
    ml = S[kStageCols + sc - 1];
    mc = S[kStageCols + sc];
    mr = S[kStageCols + sc + 1];
  }
  long long at = (long long)(y0 - 1) * nx + x;  // this lane's cell in row y
  unsigned pw = 0;  // pointer bytes of rows y-2, y-1, y in bytes 0, 1, 2
  for (int y = y0 - 1; y <= y1; ++y, at += nx) {
    int cd = 0xFF;
    const bool in = xin && y >= 0 && y < ny;
    if (!frozen) {
      const HT* Sd = S + (y + 1 - yb) * kStageCols + sc;
      const HT dl = Sd[-1], dc = Sd[0], dr = Sd[1];
      if (in) {
        if (xperim || y == 0 || y == ny - 1) {
          cd = kEdge;
        } else {
          const HT v[8] = {ul, uc, ur, ml, mr, dl, dc, dr};
          cd = receiver_from(mc, v, st);
        }
        if (own && y >= y0 && y < y1 && in_bounds(st, at, (long long)nx * ny))
          code[at] = (uint8_t)cd;
      }
      ul = ml; uc = mc; ur = mr;
      ml = dl; mc = dc; mr = dr;
    } else if (in) {
      cd = code[at];
    }
    pw = ((pw >> 8) & 0xFFFFu) | (pointer_bits(cd) << 16);
    const unsigned pl = __shfl_up_sync(0xffffffffu, pw, 1);
    const unsigned pr = __shfl_down_sync(0xffffffffu, pw, 1);
    if (own && y > y0 && y <= y1 && in_bounds(st, at - nx, (long long)nx * ny))
      mask[at - nx] = (uint8_t)mask_from_pointers(pl, pw, pr);
  }
}

template <typename HT, typename CT>
__device__ __noinline__ bool phase_codes(const StepArgs<HT, CT>& a) {
  static_assert(stage_rows<HT>() * kStageCols * sizeof(HT) + 16 <= kWarpBytes,
                "strip and barrier fit the warp slice");
  const int kRows = a.strip_rows;
  constexpr int kAlign = 16 / (int)sizeof(HT);  // staged start: a 16-byte multiple
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  HT* S = reinterpret_cast<HT*>(dyn_smem + w * kWarpBytes);
  unsigned long long* bar =
      reinterpret_cast<unsigned long long*>(dyn_smem + (w + 1) * kWarpBytes - 16);
  // fields of the kernel parameter used in the loop, held in registers
  // (the code and mask stores would otherwise force reloads)
  const int nx = a.nx, ny = a.ny;
  const bool frozen = a.frozen != 0;
  const HT* const h = a.h;
  uint8_t* const code = a.code;
  uint8_t* const mask = a.mask;
  DevState* const st = a.st;
  const int nsx = (nx + kStripOut - 1) / kStripOut;
  const int units = nsx * ((ny + kRows - 1) / kRows);
  // each block takes an equal contiguous range of strips, its warps claim
  // them one at a time (the next claim issued before the current strip)
  __shared__ int s_next;
  const int G = (int)gridDim.x, b = blockIdx.x;
  const int u1 = (int)((long long)units * (b + 1) / G);
  if (threadIdx.x == 0) s_next = (int)((long long)units * b / G);
  __syncthreads();
  int u = 0;
  if (lane == 0) u = atomicAdd(&s_next, 1);
  u = __shfl_sync(0xffffffffu, u, 0);
  // TMA staging: one box load per strip, issued by lane 0, completing on the
  // warp's mbarrier (phase parity alternates per strip)
  // (the box destination must be 128-byte aligned; a warp whose slice is
  // not stages element-wise instead)
  const bool tma = a.has_tmap && !frozen && (smem_u32(S) & 127u) == 0;
  if (tma && lane == 0) mbar_init(bar, 1);
  __syncwarp();
  unsigned parity = 0;
  bool ok = true;
  while (ok && u < u1) {
    int next = 0;
    if (lane == 0) next = atomicAdd(&s_next, 1);
    const int sy = u / nsx, sx = u - sy * nsx;
    const int x0 = sx * kStripOut;  // first owned column
    const int y0 = sy * kRows;
    // staged columns start at x0 - 2 rounded down to 16 bytes
    const int xb = (x0 - 2) & ~(kAlign - 1), yb = y0 - 2;
    if (tma) {
      if (lane == 0) {
        fence_proxy_async_smem();  // the previous strip's reads of S come first
        mbar_expect_tx(bar, (unsigned)((kRows + 4) * kStageCols * sizeof(HT)));
        tma_load_2d(S, &a.tmap, xb, yb, bar);
        if (next < u1) {
          // the warp's next strip, into L2 while this one is computed
          const int nsy = next / nsx, nsx0 = (next - nsy * nsx) * kStripOut;
          tma_prefetch_2d(&a.tmap, (nsx0 - 2) & ~(kAlign - 1), nsy * kRows - 2);
        }
      }
      ok = __all_sync(0xffffffffu, mbar_wait(bar, parity, st));
      parity ^= 1u;
      if (!ok) break;
    } else if (!frozen) {
      stage_strip(h, nx, ny, xb, yb, kRows + 4, S, lane);
    }
    codes_strip(S, code, mask, nx, ny, x0, y0, kRows, xb, frozen, lane, st);
    __syncwarp();  // S is restaged by the next unit
    u = __shfl_sync(0xffffffffu, next, 0);
  }
  __syncwarp();
  if (tma && lane == 0 && ok) mbar_inval(bar);
  __syncthreads();  // the trace marks the whole block's end of Alg 1
  trace_point(a.st, kTrLocal + 1);
  if (!grid_barrier(a.st, gridDim.x)) return false;
  trace_point(a.st, kTrCodes);
  return true;
}

// The codes of cells c .. c+3 (c a multiple of 4) as one word, bytes beyond
// the nv cells in range zero.
__device__ __forceinline__ unsigned code_word(const uint8_t* code, int c, int nv) {
  if (nv >= 4) return *reinterpret_cast<const unsigned*>(code + c);
  unsigned w = 0;
  for (int i = 0; i < nv; ++i) w |= (unsigned)code[c + i] << (8 * i);
  return w;
}

// Algs 1-2 and level 0 of Alg 3 (the stage calls and the device-wide form):
// the codes pass of the tiered step (TMA-staged strips, phase_codes) writes
// the codes and donor masks; then the cells without receiver are listed in
// ascending address order as level 0, each warp counting and then listing
// its contiguous range.  Returns false if a barrier was abandoned.
template <typename HT, typename CT>
__device__ __noinline__ bool phase_receivers(const StepArgs<HT, CT>& a, Shared& s) {
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int N = a.N;
  if (!phase_codes(a)) return false;  // ends with a grid barrier
  int w0, w1;
  warp_range(N, (int)G, b, w, &w0, &w1);
  // the count of cells without receiver (code >= 8), per warp; four cells per
  // lane per round (w0 is a multiple of 4)
  int wcnt = 0;
  for (int base = w0; base < w1; base += 128) {
    const int c = base + 4 * lane;
    const int nv = max(0, min(4, w1 - c));
    const unsigned valid = nv >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nv)) - 1u);
    wcnt += __popc(__vcmpgeu4(code_word(a.code, c, nv), 0x08080808u) & valid) >> 3;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wcnt += __shfl_down_sync(0xffffffffu, wcnt, o);
  if (lane == 0) s.wcount[w] = wcnt;
  __syncthreads();
  if (t == 0) {
    int tot = 0;
    for (int i = 0; i < kWarps; ++i) tot += s.wcount[i];
    a.partial[b] = tot;
  }
  trace_point(a.st, kTrLocal + 2);
  if (!grid_barrier(a.st, G)) return false;

  int prefix, total;
  block_prefix_of_partials<kBD>(a.partial, (int)G, b, &prefix, &total, s.sum);
  int wpre = 0;
  for (int i = 0; i < w; ++i) wpre += s.wcount[i];
  // the cells without receiver, ascending, as level 0
  {
    int run = wpre;
    for (int base = w0; base < w1; base += 128) {
      const int c = base + 4 * lane;
      const int nv = max(0, min(4, w1 - c));
      const unsigned valid = nv >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nv)) - 1u);
      const unsigned f = __vcmpgeu4(code_word(a.code, c, nv), 0x08080808u) & valid;
      const int cnt = __popc(f) >> 3;
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int pos = run + incl - cnt;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if ((f >> (8 * i)) & 1u) {
          if (in_bounds(a.st, prefix + pos, N)) a.queue[prefix + pos] = c + i;
          ++pos;
        }
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (b == 0 && t == 0) {
    a.levels[0] = 0;
    a.levels[1] = total;
  }
  __syncthreads();
  trace_point(a.st, kTrLocal + 3);
  if (!grid_barrier(a.st, G)) return false;
  trace_point(a.st, kTrLevel0);
  return true;
}

// ---- phase: device-wide Alg 3 ----------------------------------------------------

// Level 0 is queue[0, hi0).  Returns the number of levels L, or -1 if a
// barrier was abandoned or (check_all) the receiver graph left cells
// unreached (a cycle; recorded as kErrInval).
// With max_levels, returns -2 (and stops) once that many levels have been
// expanded without reaching the end (the pointer-jumping tier takes over).
template <typename HT, typename CT>
__device__ __noinline__ int phase_global_levels(const StepArgs<HT, CT>& a, Shared& s, int hi0,
                                                bool check_all, int max_levels = 0x7FFFFFFF) {
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, t = threadIdx.x;
  const int nx = a.nx;
  int lo = 0, hi = hi0, l = 0;
  while (true) {
    const int S = hi - lo;
    if (S <= kNarrowBfs) {
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
            const int ex = block_exclusive_scan<kBD>(__popc(msk), &tot, s.scan);
            if (msk && in_bounds(a.st, run + ex + __popc(msk) - 1, a.N))
              emit_donors(a.queue, run + ex, c, msk, nx);
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
          if (hi - lo > kNarrowBfs || l >= max_levels) break;
        }
        if (t == 0) {
          a.st->bfs_lo = lo;
          a.st->bfs_hi = hi;
          a.st->bfs_level = l;
          a.st->bfs_done = done ? 1 : 0;
        }
      }
      if (!grid_barrier(a.st, G)) return -1;
      trace_point(a.st, kTrBfsNarrow + l);
      lo = ld_volatile(&a.st->bfs_lo);
      hi = ld_volatile(&a.st->bfs_hi);
      l = ld_volatile(&a.st->bfs_level);
      if (ld_volatile(&a.st->bfs_done)) break;
      if (l >= max_levels) return -2;
      continue;
    }
    // wide level: each block owns a contiguous chunk of the frontier;
    // every thread takes kItems consecutive entries per round.
    const int chunk = (S + (int)G - 1) / (int)G;
    const int j0 = min(hi, lo + b * chunk), j1 = min(hi, j0 + chunk);
    long long nd = 0;
    for (int base = j0 + kItems * t; base < j1; base += kItems * kBD) {
      int cs[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) cs[i] = (base + i < j1) ? a.queue[base + i] : -1;
#pragma unroll
      for (int i = 0; i < kItems; ++i) nd += (cs[i] >= 0) ? __popc(a.mask[cs[i]]) : 0;
    }
    nd = block_sum<kBD>(nd, s.sum);
    if (t == 0) a.partial[b] = (int)nd;
    if (!grid_barrier(a.st, G)) return -1;
    int prefix, total;
    block_prefix_of_partials<kBD>(a.partial, (int)G, b, &prefix, &total, s.sum);
    int run = hi + prefix;
    for (int base0 = j0; base0 < j1; base0 += kItems * kBD) {
      const int base = base0 + kItems * t;
      int cs[kItems], ms[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) cs[i] = (base + i < j1) ? a.queue[base + i] : -1;
      int mine = 0;
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        ms[i] = (cs[i] >= 0) ? a.mask[cs[i]] : 0;
        mine += __popc(ms[i]);
      }
      int tot;
      int pos = run + block_exclusive_scan<kBD>(mine, &tot, s.scan);
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        if (ms[i] && in_bounds(a.st, pos + __popc(ms[i]) - 1, a.N)) {
          emit_donors(a.queue, pos, cs[i], ms[i], nx);
          pos += __popc(ms[i]);
        }
      }
      run += tot;
    }
    if (b == 0 && t == 0) a.levels[l + 2] = hi + total;
    if (!grid_barrier(a.st, G)) return -1;
    trace_point(a.st, kTrBfsWide + l);
    if (total == 0) break;
    lo = hi;
    hi = hi + total;
    ++l;
    if (l >= max_levels) return -2;
  }
  // L = l + 1 levels; every cell must have been reached
  const int L = l + 1;
  if (b == 0 && t == 0) a.st->nlevels = L;
  if (check_all && a.levels[L] != a.N) {
    if (b == 0 && t == 0) set_error(a.st, kErrInval);
    return -1;
  }
  return L;
}

// ---- phase: device-wide Alg 4 ----------------------------------------------------
template <typename HT, typename CT>
__device__ __noinline__ bool phase_global_accumulate(const StepArgs<HT, CT>& a, int L) {
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, t = threadIdx.x;
  const int gtid = b * kBD + t, gstride = (int)G * kBD;
  int l = L - 1;
  while (l >= 0) {
    int lo = a.levels[l], hi = a.levels[l + 1];
    if (hi - lo <= kNarrowSweep) {
      int ll = l;
      if (b == 0) {
        while (ll >= 0) {
          lo = a.levels[ll];
          hi = a.levels[ll + 1];
          if (hi - lo > kNarrowSweep) break;
          for (int j = lo + t; j < hi; j += kBD) {
            const int c = a.queue[j];
            a.cnt[c] = donor_sum(a.cnt, c, a.mask[c], a.nx);
          }
          __syncthreads();
          --ll;
        }
      } else {
        while (ll >= 0 && a.levels[ll + 1] - a.levels[ll] <= kNarrowSweep) --ll;
      }
      if (!grid_barrier(a.st, G)) return false;
      trace_point(a.st, kTrAccNarrow + ll + 1);
      l = ll;
      continue;
    }
    for (int base = lo + gtid; base < hi; base += kItems * gstride) {
      int cs[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const int j = base + i * gstride;
        cs[i] = (j < hi) ? a.queue[j] : -1;
      }
      accumulate_items(a, cs);
    }
    if (!grid_barrier(a.st, G)) return false;
    trace_point(a.st, kTrAccWide + l);
    --l;
  }
  return true;
}

// ---- phase: device-wide Algs 5-6 ---------------------------------------------------
// kNewton: Alg 6's Newton iteration for a general slope exponent
// (erode_newton) in place of the n = 1 closed form.
template <typename HT, typename CT, bool kNewton = false>
__device__ __noinline__ bool phase_global_erode(const StepArgs<HT, CT>& a, int L) {
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, t = threadIdx.x;
  const int gtid = b * kBD + t, gstride = (int)G * kBD;
  for (int j = gtid; j < a.levels[1]; j += gstride) uplift_sink(a, a.queue[j]);
  // the factors of counts beyond the tables, ahead of the sweep, so that no
  // level waits on their powers and divisions: stored by cell in the block
  // tier's queue storage (at least nx*ny doubles, idle by now)
  // (only for sweeps deep enough to pay for the pass over every count)
  double* gbig = nullptr;
  if (!kNewton && L > 64) {
    gbig = reinterpret_cast<double*>(a.pq);
    for (int j = a.levels[1] + gtid; j < a.levels[L]; j += gstride) {
      const int c = a.queue[j];
      const CT n = a.cnt[c];
      if (n >= (CT)kTableN) gbig[c] = big_count_g(a, n, nbr_diag(a.code[c]));
    }
  }
  if (!grid_barrier(a.st, G)) return false;
  trace_point(a.st, kTrUplift);
  int l = 1;
  while (l < L) {
    int lo = a.levels[l], hi = a.levels[l + 1];
    if (hi - lo <= kNarrowSweep) {
      int ll = l;
      if (b == 0) {
        while (ll < L) {
          lo = a.levels[ll];
          hi = a.levels[ll + 1];
          if (hi - lo > kNarrowSweep) break;
          for (int j = lo + t; j < hi; j += kBD) {
            int cs[kItems] = {a.queue[j], -1, -1, -1};
            erode_items<kNewton>(a, cs, gbig);
          }
          __syncthreads();
          ++ll;
        }
      } else {
        while (ll < L && a.levels[ll + 1] - a.levels[ll] <= kNarrowSweep) ++ll;
      }
      if (!grid_barrier(a.st, G)) return false;
      trace_point(a.st, kTrEroNarrow + ll);
      l = ll;
      continue;
    }
    for (int base = lo + gtid; base < hi; base += kItems * gstride) {
      int cs[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const int j = base + i * gstride;
        cs[i] = (j < hi) ? a.queue[j] : -1;
      }
      erode_items<kNewton>(a, cs, gbig);
    }
    if (!grid_barrier(a.st, G)) return false;
    trace_point(a.st, kTrEroWide + l);
    ++l;
  }
  return true;
}

// ---- block tier: Algs 3-6 on a block-private queue -----------------------------------
// Level 0 is pq[0, n0) of this block's region, with the entries' donor masks
// in pqm and receiver codes in pqk.  Returns the number of cells handled, or
// -1 if the forest outgrows the region (pcap entries, kMaxPrivLevels levels);
// then nothing was eroded.  Block barriers only.
template <typename HT, typename CT, bool kNewton = false>
__device__ __noinline__ int private_forest(const StepArgs<HT, CT>& a, Shared& s, int n0) {
  const int b = blockIdx.x, t = threadIdx.x;
  const int nx = a.nx;
  int* pq = a.pq + (size_t)b * a.pcap;
  uint8_t* pqm = a.pqm + (size_t)b * a.pcap;
  uint8_t* pqk = a.pqk + (size_t)b * a.pcap;
  int* pqf = a.pqf + (size_t)b * a.pcap;
  extern __shared__ __align__(128) unsigned char dyn_smem[];
  int* stage_q = reinterpret_cast<int*>(dyn_smem);
  uint8_t* stage_k = dyn_smem + sizeof(int) * kStage;
  int* plev = reinterpret_cast<int*>(dyn_smem + kPlevOffset);  // level offsets
  // Alg 3 on this block's trees.  Each entry carries its donor mask and its
  // receiver code, written when it is emitted, so later levels and sweeps
  // read them in queue order instead of gathering them.
  bool ovf = n0 > a.pcap;
  int lo = 0, hi = n0, PL = 1;
  if (t == 0) {
    plev[0] = 0;
    plev[1] = n0;
  }
  while (!ovf && lo < hi) {
    int run = hi;
    // Order within a private level is free (its cells are independent), so
    // thread t takes the strided entries base + i*kBD + t, i < kPItems: the
    // entry loads coalesce and all kPItems mask gathers are in flight at once.
    for (int base = lo; base < hi; base += kPItems * kBD) {
      int cs[kPItems], ms[kPItems];
#pragma unroll
      for (int i = 0; i < kPItems; ++i) {
        const int j = base + i * kBD + t;
        cs[i] = (j < hi) ? pq[j] : -1;
      }
      if (lo == 0) {
#pragma unroll
        for (int i = 0; i < kPItems; ++i) ms[i] = (cs[i] >= 0) ? pqm[base + i * kBD + t] : 0;
      } else {
        // gather this level's masks and keep them beside the entries for the
        // accumulation sweep
#pragma unroll
        for (int i = 0; i < kPItems; ++i) ms[i] = (cs[i] >= 0) ? a.mask[cs[i]] : 0;
#pragma unroll
        for (int i = 0; i < kPItems; ++i)
          if (cs[i] >= 0) pqm[base + i * kBD + t] = (uint8_t)ms[i];
      }
      // Output offsets in parent order: entry base + i*kBD + t is the
      // (i*kBD + t)-th parent of the round, so the next level keeps this
      // level's order and donors of neighbouring cells stay neighbours.
      // Each warp scans its 32 lanes per slot i; warp 0 then scans the
      // kPItems*kWarps (slot, warp) chunk totals.
      const int lane = t & 31, w = t >> 5;
      int pos_i[kPItems];
#pragma unroll
      for (int i = 0; i < kPItems; ++i) {
        const int cnt = __popc(ms[i]);
        int x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        pos_i[i] = x - cnt;
        if (lane == 31) s.chunk[i * kWarps + w] = x;
      }
      __syncthreads();
      if (w == 0) {
        int v[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          v[q] = s.chunk[lane * 8 + q];
          sum += v[q];
        }
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) s.chunk_total = x;
        int acc = x - sum;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          s.chunk[lane * 8 + q] = acc;
          acc += v[q];
        }
      }
      __syncthreads();
      const int tot = s.chunk_total;
#pragma unroll
      for (int i = 0; i < kPItems; ++i) pos_i[i] += run + s.chunk[i * kWarps + w];
      __syncthreads();  // chunk[] is rewritten by the next round
      if (run + tot > a.pcap) {
        ovf = true;
        break;
      }
      // each entry's donors are emitted contiguously; remember where they
      // start.  The emitted entries are staged in shared memory so that the
      // queue is written with coalesced stores.
      const bool staged = tot <= kStage;
#pragma unroll
      for (int i = 0; i < kPItems; ++i) {
        int pos = pos_i[i];
        if (cs[i] >= 0) pqf[base + i * kBD + t] = pos;
        int msk = ms[i];
        while (msk) {
          const int k = __ffs(msk) - 1;
          msk &= msk - 1;
          const int d = cs[i] + nbr_off(k, nx);
          if (staged) {
            stage_q[pos - run] = d;
            stage_k[pos - run] = (uint8_t)(7 - k);
          } else {
            pq[pos] = d;
            pqk[pos] = (uint8_t)(7 - k);
          }
          ++pos;
        }
      }
      if (staged) {
        __syncthreads();
        for (int o = t; o < tot; o += kBD) {
          pq[run + o] = stage_q[o];
          pqk[run + o] = stage_k[o];
        }
        __syncthreads();
      }
      run += tot;
    }
    __syncthreads();
    trace_point(a.st, kTrLocal + 0x1000 + PL);  // block 0: private level PL-1 expanded
    if (ovf || run == hi) break;
    if (PL >= a.priv_levels) {
      ovf = true;
      break;
    }
    ++PL;
    if (t == 0) plev[PL] = run;
    lo = hi;
    hi = run;
  }
  if (ovf) return -1;

  // Alg 4 in queue order, this block's levels from the highest down to level
  // 1 (a time step needs the counts of eroding cells only): an entry's count
  // is 1 plus the counts of its donors, which sit contiguously at
  // [pqf, pqf + number of donors) in the next level.
  CT* cntq = a.cntq + (size_t)b * a.pcap;
  for (int l = PL - 1; l >= 1; --l) {
    const int l0 = plev[l], l1 = plev[l + 1];
    for (int base = l0 + t; base < l1; base += kItems * kBD) {
      int fs[kItems], ns[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const int j = base + i * kBD;
        fs[i] = (j < l1) ? pqf[j] : 0;
        ns[i] = (j < l1) ? __popc(pqm[j]) : 0;
      }
      CT sum[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        sum[i] = 1;
        for (int q = 0; q < ns[i]; ++q) sum[i] += cntq[fs[i] + q];
      }
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const int j = base + i * kBD;
        if (j < l1) cntq[j] = sum[i];
      }
    }
    __syncthreads();
    trace_point(a.st, kTrLocal + 0x2000 + l);  // block 0: private level l accumulated
  }
  trace_point(a.st, kTrPrivAcc);
  // Alg 5 on level 0 (pits only), then Alg 6 from level 1 up
  for (int j = t; j < plev[1]; j += kBD)
    if (pqk[j] == kSink) {
      const int c = pq[j];
      if constexpr (sizeof(HT) == 8) {
        a.h[c] = __dadd_rn(a.h[c], uplift_dt(a, c));
      } else {
        a.h[c] = __fadd_rn(a.h[c], uplift_dt_f(a, c));
      }
    }
  __syncthreads();
  for (int l = 1; l < PL; ++l) {
    const int l0 = plev[l], l1 = plev[l + 1];
    for (int base = l0 + t; base < l1; base += kItems * kBD) {
      int cs[kItems], ks[kItems];
      CT ns[kItems];
      HT hc[kItems], hr[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const int j = base + i * kBD;
        cs[i] = (j < l1) ? pq[j] : -1;
        ks[i] = (j < l1) ? pqk[j] : 0;
        ns[i] = (j < l1) ? cntq[j] : 1;
      }
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        if (cs[i] >= 0) {
          hc[i] = a.h[cs[i]];
          hr[i] = a.h[cs[i] + nbr_off(ks[i], nx)];
        }
      }
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        if (cs[i] >= 0) {
          if (!in_bounds(a.st, cs[i], a.N)) continue;
          if constexpr (kNewton) {
            a.h[cs[i]] = erode_newton(a, cs[i], ks[i], ns[i], hc[i], hr[i]);
          } else {
            a.h[cs[i]] = erode_value(a, cs[i], ks[i], ns[i], hc[i], hr[i]);
          }
        }
      }
    }
    __syncthreads();
  }
  return plev[PL];
}

}  // namespace lem

#include "lem_tiles.cuh"
#include "lem_jump.cuh"

namespace lem {

// kNewton: Alg 6 for a general slope exponent (newton_solve) in every tier
// in place of the n = 1 closed form.
template <typename HT, typename CT, bool kNewton = false>
__global__ void __launch_bounds__(kBD, 1) lem_step_kernel(const __grid_constant__ StepArgs<HT, CT> a) {
  __shared__ Shared s;
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  if ((a.phases & kPhTiles) && lead) {
    a.st->dev_roots[0] = a.st->dev_roots[1] = 0;
    a.st->ovf_count[0] = a.st->ovf_count[1] = 0;
    a.st->covered[0] = a.st->covered[1] = 0;
  }

  for (int step = 0; step < a.nsteps; ++step) {
    trace_point(a.st, kTrStart + step);
    if (a.phases & kPhTiles) {
      // the tiered step: Alg 1, a grid barrier, the warp and block tiers, a
      // grid barrier, and the device tier only if some roots reached it
      const int par = step & 1;
      if (!phase_codes(a)) return;
      // an error found by Alg 1 (a non-finite elevation) stops the step before
      // any elevation changes (every block reads the word after the barrier)
      if (ld_volatile(&a.st->err) != 0) return;
      if (lead) {
        // every block has left the previous step, the last reader of these
        a.st->dev_roots[par ^ 1] = 0;
        a.st->ovf_count[par ^ 1] = 0;
        a.st->covered[par ^ 1] = 0;
      }
      // the warp tier; overflowed items are listed in levels[] (idle until
      // the device tier)
      phase_tiles<HT, CT, kNewton>(a, s, &a.st->tiles_next[par], &a.st->ovf_count[par],
                                   a.levels, &a.st->covered[par]);
      if (!grid_barrier(a.st, gridDim.x)) return;
      trace_point(a.st, kTrTilesEnd);
      if (lead) a.st->tiles_next[par] = 0;  // every block has stopped claiming
      const int n_ovf = ld_volatile(&a.st->ovf_count[par]);
      if (n_ovf > 0) {
        phase_block_tier<HT, CT, kNewton>(a, s, n_ovf, a.levels, &a.st->dev_roots[par],
                                          &a.st->covered[par]);
        if (!grid_barrier(a.st, gridDim.x)) return;
        trace_point(a.st, kTrBlockEnd);
      }
      const int dr = ld_volatile(&a.st->dev_roots[par]);
      if (dr > 0) {
        // breadth-first levels first, unless the last device tier was deep;
        // beyond jump_cap levels the pointer-jumping tier takes the trees
        const bool can_jump = !kNewton && a.jt != nullptr;
        int L = -2;
        if (!can_jump || ld_volatile(&a.st->jump_hint) == 0) {
          if (lead) {
            a.levels[0] = 0;
            a.levels[1] = dr;
          }
          L = phase_global_levels(a, s, dr, false, can_jump ? a.jump_cap : 0x7FFFFFFF);
          if (L == -1) return;
        }
        if (L == -2) {
          if (phase_jump(a, s, dr) < 0) return;  // ends with a grid barrier
          if (lead) {
            const unsigned long long cells = a.st->jump_step_cells + (unsigned long long)dr;
            a.st->covered[par] += (int)cells;
            a.st->tier_cells[2] += cells;
            a.st->global_steps += 1;
            a.st->jump_steps += 1;
            // stay with jumping while the paths are longer than the cap
            const int r = min(max(a.st->jump_rounds - 1, 0), 62);
            a.st->jump_hint = (1LL << r) > (long long)a.jump_cap ? 1 : 0;
          }
        } else {
          if (!phase_global_accumulate(a, L)) return;
          if (!phase_global_erode<HT, CT, kNewton>(a, L)) return;  // ends with a grid barrier
          if (lead) {
            a.st->covered[par] += a.levels[L];
            a.st->tier_cells[2] += (unsigned long long)a.levels[L];
            a.st->global_steps += 1;
            a.st->jump_hint = 0;
          }
        }
      } else if (lead) {
        a.st->private_steps += 1;
      }
      // every cell lies in exactly one tree unless a frozen graph has a cycle
      if (lead && ld_volatile(&a.st->covered[par]) != a.N) set_error(a.st, kErrInval);
      continue;
    }

    if (a.phases & kPhRec)
      if (!phase_receivers(a, s)) return;
    int L = -1;
    if (a.phases & kPhLev) {
      L = phase_global_levels(a, s, a.levels[1], true);
      if (L < 0) return;
    }
    if (a.phases & (kPhAcc | kPhEro)) {
      if (L < 0) L = ld_volatile(&a.st->nlevels);
      if ((a.phases & kPhAcc) && !phase_global_accumulate(a, L)) return;
      if ((a.phases & kPhEro) && !phase_global_erode<HT, CT, kNewton>(a, L)) return;
    }
  }
}

}  // namespace lem
