// lem_context.cuh -- the context behind the opaque lem_ctx handle of
// include/lem.h: parameters, the caller's bound buffers and the library's own
// device scratch.  Shared by the C-ABI translation units.
#pragma once

#include "lem.h"
#include "lem_step_kernel.cuh"

struct lem_ctx {
  // parameters and bound caller buffers
  lem_params p;
  int N = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  void* h = nullptr;
  const double* Uf = nullptr;
  uint8_t* code = nullptr;       // code_base + kCodeGuard
  uint8_t* code_base = nullptr;  // allocation with guard bytes
  uint8_t* mask = nullptr;
  int* queue = nullptr;
  int* levels = nullptr;
  void* cnt = nullptr;
  double2* Ftab = nullptr;  // {F, F/(1+F)} by count (lem_step_kernel.cuh)
  double2* Gtab = nullptr;  // {dt*A^m/dx, dt*A^m/(dx*sqrt2)} = dF/dK by count
  float* gtab = nullptr;
  lem::DevState* st = nullptr;
  int* partial = nullptr;
  int* pq = nullptr;  // block-private queues, pcap entries per block
  uint8_t* pqm = nullptr;  // donor mask per private-queue entry
  uint8_t* pqk = nullptr;  // receiver code per private-queue entry
  int* pqf = nullptr;      // first-donor position per private-queue entry
  void* cntq = nullptr;    // counts in private-queue order
  int pcap = 0;
  int mode = 0;       // 0: block-private levels with fallback, 1: device-wide only
  int strip_rows = 0; // lem_set_tiling: rows per strip of the codes pass (0: heuristic)
  int half_tiles = 0; // lem_set_tiling: warp tier on half-height tiles
  int grid = 0;
  int* host_status = nullptr;  // pinned: [err, nlevels]
  bool rec_valid = false, lev_valid = false, acc_valid = false, frozen = false;
  bool graph_valid = false;  // code/mask hold the graph of the last step or lem_receivers
  double Kdt = 0, dxd = 0, area_scale = 0;
  // Alg 6 for a general slope exponent (lem_set_slope_exponent); 0 updates =
  // the n = 1 closed form
  int newton_iters = 0;
  double nexp = 1.0, neps = 0.0, dxn = 0.0, dxdn = 0.0, dfac = 0.0, dfacd = 0.0;
  // depression filling (lem_fill.cu): scratch allocated by the first flood
  int fill_on = 0;             // lem_step floods before every step
  int fill_grid = 0;           // co-resident blocks of the flood kernel
  void* fill_w = nullptr;      // relaxed surface, nx*ny elements
  uint8_t* fill_dirty = nullptr;  // two per-tile flag arrays
  int* fill_ptr = nullptr;     // chain pointers, nx*ny
  // flow accumulation with multiple flow directions (lem_mfd.cu): scratch
  // allocated by the first call
  int mfd_grid = 0;
  int* mfd_pending = nullptr;  // donors not yet computed, nx*ny
  double* mfd_norm = nullptr;  // receivers' sum of slope^p, nx*ny
  int* mfd_queue = nullptr;    // the levels, nx*ny
  void* mfd_state = nullptr;
  void* fill_state = nullptr;  // round counters
  // the device tier's pointer-jumping form: scratch allocated by the first
  // lem_step in step mode 0 (44 bytes per cell)
  unsigned long long* jt = nullptr;  // 2 words per cell
  double2* jab1 = nullptr;
  int* jp0 = nullptr;
  int* jp1 = nullptr;
  unsigned* jstamp = nullptr;
  double wait_limit_s = 2.0;
  unsigned long long* trace = nullptr;  // device trace buffer (lem_trace_enable)
  lem::TmaDesc tmap{};      // TMA descriptor of the bound h (host copy)
  bool tmap_ok = false;     // tmap describes the bound h
};
