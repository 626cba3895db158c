// lem_jump.cuh -- Algs 3-6 for trees too deep for level-by-level sweeps.
//
// Included by lem_step_kernel.cuh after the device-wide phases.
//
// The paper's level order needs one device-wide synchronisation per level
// (Section "The Algorithm", Alg 3, and the discussion of barriers); a tree
// whose flow paths are thousands of cells long makes that a sequence of
// thousands of short, latency-bound steps.  This tier instead reaches the
// same per-cell results in O(log depth) device-wide rounds, by pointer
// jumping over every cell of the grid:
//
//  * Alg 4 (counts): the Euler tour of each receiver tree -- enter a cell,
//    visit its donors in k order, leave it -- is a linked list whose links
//    each cell knows from its receiver code and donor mask alone.  Ranking
//    every list by pointer jumping (Wyllie) gives each tour node its
//    distance to the tour's end, and a cell's count (the size of the tree
//    above it, itself included) is (rank(enter) - rank(leave) + 1) / 2,
//    exactly.  The end of each tour (leaving the root) also names the root,
//    which tells the cells of the trees handed to this tier apart.
//  * Algs 5-6 (uplift, implicit erosion with n-hat = 1): each eroding cell's
//    new elevation is affine in its receiver's, h'_c = (1 - g_c) h0_c +
//    g_c h'_r (g = F/(1+F), h0 = h + dt U), and a root's is known (h + dt U
//    for a pit, h on the perimeter).  Composing the maps along the receiver
//    pointers -- (A, B, p) <- (A + B A_p, B B_p, p_p), h'_c = A + B h'_p --
//    halves every remaining path per round.  The sum runs in FP64 for either
//    elevation type: its terms are the path's elevations weighted by
//    non-negative weights that sum to one, so it is within a few units in
//    the last place of the sequential sweep (no cancellation beyond that of
//    the elevations themselves), and FP32 results are rounded once.
//
// The tier handles the trees whose roots the warp and block tiers handed to
// the device-wide tier (queue[0, dr)); cells of every other tree are
// ranked (the tour covers the whole grid) but neither counted nor eroded.
// Scratch: the tour (2 words per cell), reused as the first (A, B) buffer,
// a second (A, B) buffer, two pointer buffers and a root stamp per cell.
#pragma once

namespace lem {

// Tour node ids: enter(c) = 2c, leave(c) = 2c + 1; a word holds the next
// node (low 32 bits) and the hops to it (high 32 bits).  The end of a tour
// (leaving its root) links to itself with 0 hops.
__device__ __forceinline__ unsigned long long tour_word(unsigned next, unsigned hops) {
  return (unsigned long long)hops << 32 | next;
}

// Device-wide "did anything change" vote of round r: every block that
// changed something adds 1 to word r % 3; the total is read by every block
// after a grid barrier (-1 if the barrier was abandoned).  Block 0 then
// clears the word of round r + 2: every block has read it (round r - 1)
// before arriving at this barrier, and none writes it before the next
// barrier.  The three words must be zero before round 0.
__device__ __forceinline__ int round_vote(DevState* st, int r, int mine, int* s_any) {
  __syncthreads();
  if (threadIdx.x == 0) *s_any = 0;
  __syncthreads();
  if (mine) atomicOr(s_any, 1);
  __syncthreads();
  if (threadIdx.x == 0 && *s_any) atomicAdd(&st->jump_vote[r % 3], 1);
  if (!grid_barrier(st, gridDim.x)) return -1;
  const int v = ld_volatile(&st->jump_vote[r % 3]);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->jump_vote[(r + 2) % 3] = 0;
  return v;
}

// Algs 3-6 for the trees rooted at queue[0, dr) by pointer jumping (see the
// file comment).  The number of eroding cells handled is left in
// st->jump_step_cells and the erosion rounds in st->jump_rounds.  Returns
// 0, or -1 if a barrier was abandoned (or the graph has a cycle).  Ends with
// a grid barrier.
template <typename HT, typename CT>
__device__ __noinline__ long long phase_jump(const StepArgs<HT, CT>& a, Shared& s, int dr) {
  const int b = blockIdx.x, t = threadIdx.x;
  const int gtid = b * kBD + t, gstride = (int)gridDim.x * kBD;
  const int N = a.N, nx = a.nx;
  unsigned long long* const jt = a.jt;
  double2* const ab0 = reinterpret_cast<double2*>(a.jt);
  DevState* const st = a.st;
  __shared__ int s_any;
  const unsigned epoch = (unsigned)ld_volatile(&st->jump_epoch) + 1u;
  if (t < 8) s.off[t] = nbr_off(t, nx);
  __syncthreads();
  // the tour's links, and the stamp of this step on the tier's roots
  for (int c = gtid; c < N; c += gstride) {
    const int cd = __ldcg(a.code + c);
    const int msk = __ldcg(a.mask + c);
    const unsigned enter_next =
        msk ? 2u * (unsigned)(c + s.off[__ffs(msk) - 1]) : 2u * (unsigned)c + 1u;
    unsigned leave_next = 2u * (unsigned)c + 1u, leave_hops = 0;
    if (cd < kSink) {
      const int p = c + s.off[cd];
      const int rest = __ldcg(a.mask + p) & (0xFE << (7 - cd)) & 0xFF;  // p's donors after c
      leave_next = rest ? 2u * (unsigned)(p + s.off[__ffs(rest) - 1]) : 2u * (unsigned)p + 1u;
      leave_hops = 1;
    }
    jt[2 * (size_t)c] = tour_word(enter_next, 1);
    jt[2 * (size_t)c + 1] = tour_word(leave_next, leave_hops);
  }
  for (int j = gtid; j < dr; j += gstride) {
    const int r = __ldcg(a.queue + j);
    if (in_bounds(st, r, N)) a.jstamp[r] = epoch;
  }
  if (b == 0 && t == 0) {
    st->jump_vote[0] = st->jump_vote[1] = st->jump_vote[2] = 0;
    st->jump_step_cells = 0;
  }
  if (!grid_barrier(st, gridDim.x)) return -1;
  trace_point(st, kTrJumpTour);
  // Wyllie's list ranking, in place: every word is a consistent (node, hops)
  // pair whenever it is read, so reading a partner's old or new word both
  // keep hops = distance to node.  Everything this tier reads that other
  // blocks wrote during the launch is loaded from L2 (__ldcg): an SM's L1 is
  // not kept coherent with other SMs' stores.
  const size_t nodes = 2 * (size_t)N;
  bool ranked = false;
  for (int round = 0; round < 64; ++round) {
    int mine = 0;
    for (size_t x = gtid; x < nodes; x += gstride) {
      const unsigned long long w = __ldcg(jt + x);
      const unsigned n = (unsigned)w;
      if (n == (unsigned)x) continue;
      if (!in_bounds(st, n, (long long)nodes)) continue;
      const unsigned long long wn = __ldcg(jt + n);
      const unsigned nn = (unsigned)wn;
      if (nn == n) continue;  // n is the end of the tour
      jt[x] = tour_word(nn, (unsigned)(w >> 32) + (unsigned)(wn >> 32));
      mine = 1;
    }
    const int v = round_vote(st, round, mine, &s_any);
    if (v < 0) return -1;
    trace_point(st, kTrJumpRank + round);
    if (v == 0) {
      ranked = true;
      break;
    }
  }
  if (!ranked) {
    // no tour ended within 64 rounds: the (frozen) graph has a cycle
    if (b == 0 && t == 0) set_error(st, kErrInval);
    return -1;
  }
  // counts and erosion factors of the tier's cells and their first (A, B,
  // p); every other cell gets p = -1 in both pointer buffers
  long long eroded = 0;
  for (int c = gtid; c < N; c += gstride) {
    const unsigned long long we = __ldcg(jt + 2 * (size_t)c);
    const unsigned long long wl = __ldcg(jt + 2 * (size_t)c + 1);
    const int root = (int)((unsigned)wl >> 1);
    if (!in_bounds(st, root, N) || __ldcg(a.jstamp + root) != epoch) {
      a.jp0[c] = -1;
      a.jp1[c] = -1;
      continue;
    }
    const int cd = __ldcg(a.code + c);
    const double hc = (double)__ldcg(a.h + c);
    double A, B;
    int p;
    if (cd >= kSink) {
      A = cd == kSink ? hc + uplift_dt(a, c) : hc;
      B = 0.0;
      p = c;
    } else {
      const CT count = (CT)(((long long)(we >> 32) - (long long)(wl >> 32) + 1) / 2);
      const bool diag = nbr_diag(cd);
      const double g = count < (CT)kTableN ? a.Ftab[(diag ? kTableN : 0) + (int)count].y
                                           : big_count_g(a, count, diag);
      const double h0 = hc + uplift_dt(a, c);
      A = __fma_rn(-g, h0, h0);
      B = g;
      p = c + s.off[cd];
      ++eroded;
    }
    ab0[c] = make_double2(A, B);  // over this cell's own two tour words
    a.jp0[c] = p;
  }
  if (b == 0 && t == 0) st->jump_vote[0] = st->jump_vote[1] = st->jump_vote[2] = 0;
  if (!grid_barrier(st, gridDim.x)) return -1;
  trace_point(st, kTrJumpInit);
  // pointer jumping on the affine maps, ping-pong between the two buffers;
  // a map whose B is zero is final (it reached its root, or the product of
  // factors below one vanished)
  int src = 0, rounds = 0;
  for (int round = 0; round < 64; ++round) {
    const double2* abs_ = src ? a.jab1 : ab0;
    double2* abd = src ? ab0 : a.jab1;
    const int* ps = src ? a.jp1 : a.jp0;
    int* pd = src ? a.jp0 : a.jp1;
    int mine = 0;
    for (int c = gtid; c < N; c += gstride) {
      int p = __ldcg(ps + c);
      if (p < 0) continue;
      double2 m = __ldcg(abs_ + c);
      if (m.y != 0.0 && in_bounds(st, p, N)) {
        const double2 q = __ldcg(abs_ + p);
        m = make_double2(__fma_rn(m.y, q.x, m.x), __dmul_rn(m.y, q.y));
        p = __ldcg(ps + p);
        mine = 1;
      }
      abd[c] = m;
      pd[c] = p;
    }
    src ^= 1;
    rounds = round + 1;
    const int v = round_vote(st, round, mine, &s_any);
    if (v < 0) return -1;
    trace_point(st, kTrJumpErode + round);
    if (v == 0) break;
  }
  {
    const double2* fin = src ? a.jab1 : ab0;
    const int* pf = src ? a.jp1 : a.jp0;
    for (int c = gtid; c < N; c += gstride)
      if (__ldcg(pf + c) >= 0) a.h[c] = (HT)__ldcg(fin + c).x;
  }
  eroded = block_sum<kBD>(eroded, s.sum);
  if (t == 0) atomicAdd(&st->jump_step_cells, (unsigned long long)eroded);
  if (b == 0 && t == 0) {
    st->jump_epoch = (int)epoch;
    st->jump_rounds = rounds;
  }
  if (!grid_barrier(st, gridDim.x)) return -1;
  return 0;
}

}  // namespace lem
