/*
 * lem_oracle.c -- serial FP64 restatement of the landscape-evolution step of
 * Barnes, "Accelerating a Landscape Evolution Model with Parallelism"
 * (arXiv:1803.02977), Section "The Algorithm", Algorithms 1-6.
 *
 * TEST INFRASTRUCTURE ONLY: the plain reference the CUDA library is checked
 * against.  Written for a reader to verify against the paper by eye; no
 * blocking, fusion or reordering beyond what the algorithms state.
 * Compile with -O2 -ffp-contract=off (no fused multiply-add, no fast-math).
 */
#include "lem_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Double nearest 1/sqrt(2) and sqrt(2); both are decimal literals so that
 * the value does not depend on a library's sqrt. */
static const double ORC_INV_SQRT2 = 0.70710678118654752440;
static const double ORC_SQRT2 = 1.41421356237309504880;

/* Offsets (dx, dy) of the eight neighbours in ascending address order. */
static const int ORC_DX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int ORC_DY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};

static int orc_is_diagonal(int k) { return ORC_DX[k] != 0 && ORC_DY[k] != 0; }

static int orc_on_perimeter(int nx, int ny, int x, int y) {
  return x == 0 || y == 0 || x == nx - 1 || y == ny - 1;
}

/* ---- Alg 1: Determine Receivers ------------------------------------------ */

static void orc_receivers_impl(int nx, int ny, const double* h, const float* hf,
                               int32_t* rec) {
  /* Initialise Rec to NoFlow (self) -- this covers the perimeter. */
  for (int64_t c = 0; c < (int64_t)nx * ny; ++c) rec[c] = (int32_t)c;
  for (int y = 1; y < ny - 1; ++y) {
    for (int x = 1; x < nx - 1; ++x) {
      int64_t c = (int64_t)y * nx + x;
      double hc = h ? h[c] : (double)hf[c];
      double smax = 0.0;     /* maximum slope so far */
      int64_t nmax = c;      /* neighbour with that slope (NoFlow = self) */
      for (int k = 0; k < 8; ++k) {
        int64_t n = (int64_t)(y + ORC_DY[k]) * nx + (x + ORC_DX[k]);
        double hn = h ? h[n] : (double)hf[n];
        double w = orc_is_diagonal(k) ? ORC_INV_SQRT2 : 1.0;
        double s = (hc - hn) * w;  /* slope from c to n, times dx */
        if (s > smax) {
          smax = s;
          nmax = n;
        }
      }
      rec[c] = (int32_t)nmax;
    }
  }
}

void orc_receivers(int nx, int ny, const double* h, int32_t* rec) {
  orc_receivers_impl(nx, ny, h, NULL, rec);
}

void orc_receivers_f32(int nx, int ny, const float* h, int32_t* rec) {
  orc_receivers_impl(nx, ny, NULL, h, rec);
}

/* ---- Alg 2: Determine Donors --------------------------------------------- */

void orc_donors_grid(int nx, int ny, const int32_t* rec, int32_t* dnum, int32_t* donor) {
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      int64_t c = (int64_t)y * nx + x;
      dnum[c] = 0;
      for (int k = 0; k < 8; ++k) {
        int xn = x + ORC_DX[k], yn = y + ORC_DY[k];
        if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
        int64_t n = (int64_t)yn * nx + xn;
        if (rec[n] == c) {
          donor[8 * c + dnum[c]] = (int32_t)n;
          dnum[c] = dnum[c] + 1;
        }
      }
    }
  }
}

int orc_donors_graph(int n, const int32_t* rec, int dmax, int32_t* dnum, int32_t* donor) {
  for (int c = 0; c < n; ++c) {
    dnum[c] = 0;
    for (int v = 0; v < n; ++v) {
      if (v != c && rec[v] == c) {
        if (dnum[c] >= dmax) return -1;
        donor[(int64_t)dmax * c + dnum[c]] = v;
        dnum[c] = dnum[c] + 1;
      }
    }
  }
  return 0;
}

/* ---- Alg 3: Generate Queue (breadth first) ------------------------------- */

int64_t orc_queue(int64_t n, const int32_t* rec, int dmax, const int32_t* dnum,
                  const int32_t* donor, int32_t* queue, int64_t* levels, int32_t* depth) {
  int64_t nqueue = 0;  /* open location in Queue */
  int64_t ls = 0;      /* write location in Levels */
  for (int64_t c = 0; c < n; ++c) depth[c] = -1;

  levels[ls++] = 0;
  /* Source cells: every cell without a receiver. */
  for (int64_t c = 0; c < n; ++c) {
    if (rec[c] == c) {
      queue[nqueue++] = (int32_t)c;
      depth[c] = 0;
    }
  }
  if (nqueue == 0) return 0;
  levels[ls++] = nqueue;

  /* Expand level by level: the donors of the cells of level l form l+1. */
  int64_t lo = 0, hi = nqueue;
  int32_t l = 0;
  while (lo < hi) {
    for (int64_t i = lo; i < hi; ++i) {
      int32_t c = queue[i];
      for (int k = 0; k < dnum[c]; ++k) {
        int32_t d = donor[(int64_t)dmax * c + k];
        queue[nqueue++] = d;
        depth[d] = l + 1;
      }
    }
    lo = hi;
    hi = nqueue;
    if (hi > lo) levels[ls++] = nqueue;  /* close the non-empty level */
    l = l + 1;
  }
  return ls - 1;
}

/* ---- Alg 4: Flow Accumulation (Eq. 2, w = 1) ----------------------------- */

void orc_accumulate(int64_t n, const int32_t* queue, const int64_t* levels, int64_t nlevels,
                    int dmax, const int32_t* dnum, const int32_t* donor, int64_t* cnt) {
  for (int64_t c = 0; c < n; ++c) cnt[c] = 1;
  for (int64_t l = nlevels - 2; l >= 0; --l) {
    for (int64_t i = levels[l]; i < levels[l + 1]; ++i) {
      int32_t c = queue[i];
      for (int k = 0; k < dnum[c]; ++k) {
        int32_t d = donor[(int64_t)dmax * c + k];
        cnt[c] = cnt[c] + cnt[d];
      }
    }
  }
}

/* ---- Alg 5: Uplift -------------------------------------------------------- */

void orc_uplift(int nx, int ny, double* h, const orc_params* p) {
  for (int y = 1; y < ny - 1; ++y) {
    for (int x = 1; x < nx - 1; ++x) {
      int64_t c = (int64_t)y * nx + x;
      double u = p->Ufield ? p->Ufield[c] : p->U;
      h[c] = h[c] + u * p->dt;
    }
  }
}

/* ---- Alg 6: Calculate Erosion -------------------------------------------- */

/* dist(c, r) for a receiver r adjacent to c. */
static double orc_dist(int nx, int32_t c, int32_t r, double dx) {
  int64_t dxi = (int64_t)(r % nx) - (int64_t)(c % nx);
  int64_t dyi = (int64_t)(r / nx) - (int64_t)(c / nx);
  return (dxi != 0 && dyi != 0) ? dx * ORC_SQRT2 : dx;
}

void orc_erode(int nx, int ny, double* h, const int32_t* rec, const int32_t* queue,
               const int64_t* levels, int64_t nlevels, const int64_t* cnt, const orc_params* p) {
  (void)ny;
  for (int64_t l = 1; l < nlevels; ++l) {
    for (int64_t i = levels[l]; i < levels[l + 1]; ++i) {
      int32_t c = queue[i];           /* focal cell */
      int32_t r = rec[c];             /* its receiver */
      double A = (double)cnt[c] * p->area_scale;
      double F = p->K * p->dt * pow(A, p->m) / orc_dist(nx, c, r, p->dx);
      double h0 = h[c];
      double hr = h[r];
      h[c] = (h0 + F * hr) / (1.0 + F);
    }
  }
}

void orc_erode_newton(int nx, int ny, double* h, const int32_t* rec, const int32_t* queue,
                      const int64_t* levels, int64_t nlevels, const int64_t* cnt,
                      const orc_params* p, double n_exp, double eps, int max_iter) {
  (void)ny;
  for (int64_t l = 1; l < nlevels; ++l) {
    for (int64_t i = levels[l]; i < levels[l + 1]; ++i) {
      int32_t c = queue[i];
      int32_t r = rec[c];
      double A = (double)cnt[c] * p->area_scale;
      double F = p->K * p->dt * pow(A, p->m) / pow(orc_dist(nx, c, r, p->dx), n_exp);
      double h0 = h[c];
      double hn = h[r];
      /* (h - h_r)^n-hat is undefined below the receiver for non-integer
       * n-hat: a cell whose uplifted elevation is not above its receiver's
       * new elevation keeps it (no erosion without a downhill slope). */
      if (!(h0 - hn > 0.0)) continue;
      double hnew = h0;      /* current updated value */
      double hp = h0;        /* previous updated value */
      double delta = 2.0 * eps;
      int it = 0;
      while (fabs(delta) > eps && it < max_iter) {
        double f = hnew - h0 + F * pow(hnew - hn, n_exp);
        double fp = 1.0 + F * n_exp * pow(hnew - hn, n_exp - 1.0);
        hnew = hnew - f / fp;
        delta = hnew - hp;
        hp = hnew;
        ++it;
      }
      h[c] = hnew;
    }
  }
}

/* ---- Multiple flow directions (Section "Multiple Flow Directions"; Eq. 2) - */
/* Receivers of an interior cell: every strictly lower neighbour.  Its flow
 * is split in proportion to slope^p (slope = (h_c - h_n) * w_k as in Alg 1),
 * alpha(c -> n_k) = s_k^p / sum over receivers of s^p, the sum taken in k
 * order.  Flow accumulation (Eq. 2): A(c) = w(c) + sum over the donors n of
 * c, in k order of c's neighbours, of alpha(n -> c) * A(n), computed once
 * every donor of c is final (cells taken level by level from those without
 * donors). */

static double orc_mfd_slope(const double* h, int64_t c, int64_t n, int k) {
  double d = h[c] - h[n];
  return orc_is_diagonal(k) ? d * ORC_INV_SQRT2 : d;
}

/* sum over c's receivers of slope^p, 0 without receivers */
static double orc_mfd_norm(int nx, int ny, const double* h, int64_t c, double p) {
  int x = (int)(c % nx), y = (int)(c / nx);
  if (orc_on_perimeter(nx, ny, x, y)) return 0.0;
  double sum = 0.0;
  for (int k = 0; k < 8; ++k) {
    int64_t n = (int64_t)(y + ORC_DY[k]) * nx + (x + ORC_DX[k]);
    if (h[n] < h[c]) {
      double s = orc_mfd_slope(h, c, n, k);
      sum = sum + (p == 1.0 ? s : pow(s, p));
    }
  }
  return sum;
}

int64_t orc_accumulate_mfd(int nx, int ny, const double* h, const double* w, double p,
                           double* A, int32_t* level) {
  int64_t n = (int64_t)nx * ny;
  int32_t* pending = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t* frontier = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  double* norm = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!pending || !frontier || !norm) {
    free(pending);
    free(frontier);
    free(norm);
    return -1;
  }
  /* donors of c: interior neighbours strictly above it */
  for (int64_t c = 0; c < n; ++c) {
    int x = (int)(c % nx), y = (int)(c / nx);
    int cntd = 0;
    for (int k = 0; k < 8; ++k) {
      int xn = x + ORC_DX[k], yn = y + ORC_DY[k];
      if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
      if (orc_on_perimeter(nx, ny, xn, yn)) continue;
      if (h[(int64_t)yn * nx + xn] > h[c]) ++cntd;
    }
    pending[c] = cntd;
    norm[c] = orc_mfd_norm(nx, ny, h, c, p);
  }
  /* level 0: cells without donors, ascending address */
  int64_t head = 0, tail = 0;
  for (int64_t c = 0; c < n; ++c)
    if (pending[c] == 0) {
      frontier[tail++] = c;
      if (level) level[c] = 0;
    }
  int64_t nlevels = 0;
  while (head < tail) {
    int64_t end = tail;
    ++nlevels;
    for (; head < end; ++head) {
      int64_t c = frontier[head];
      int x = (int)(c % nx), y = (int)(c / nx);
      /* Eq. 2, pulled from the donors in k order */
      double a = w ? w[c] : 1.0;
      for (int k = 0; k < 8; ++k) {
        int xn = x + ORC_DX[k], yn = y + ORC_DY[k];
        if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
        if (orc_on_perimeter(nx, ny, xn, yn)) continue;
        int64_t d = (int64_t)yn * nx + xn;
        if (!(h[d] > h[c])) continue;
        /* the slope of the donor toward c: c is neighbour 7-k of d */
        double s = orc_mfd_slope(h, d, c, 7 - k);
        double alpha = (p == 1.0 ? s : pow(s, p)) / norm[d];
        a = a + alpha * A[d];
      }
      A[c] = a;
      /* release the receivers */
      if (!orc_on_perimeter(nx, ny, x, y)) {
        for (int k = 0; k < 8; ++k) {
          int64_t r = (int64_t)(y + ORC_DY[k]) * nx + (x + ORC_DX[k]);
          if (h[r] < h[c] && --pending[r] == 0) {
            frontier[tail++] = r;
            if (level) level[r] = (int32_t)nlevels;
          }
        }
      }
    }
  }
  free(pending);
  free(frontier);
  free(norm);
  return nlevels;
}

/* ---- Depression filling before receivers (Section "Local Minima") -------- */
/* Priority-Flood with epsilon increments: cells leave one priority queue in
 * order of their filled elevation w (ties by address), starting from the
 * perimeter at w = h; each neighbour n seen for the first time gets
 * w[n] = max(h[n], next representable value above w[c]) and joins the
 * queue.  One queue for every cell keeps the pops in non-decreasing w, so a
 * cell's first w is its least one. */

typedef struct {
  double w;
  int64_t c;
} orc_pq_item;

static int orc_pq_less(const orc_pq_item* a, const orc_pq_item* b) {
  return a->w < b->w || (a->w == b->w && a->c < b->c);
}

static void orc_pq_push(orc_pq_item* q, int64_t* n, orc_pq_item it) {
  int64_t i = (*n)++;
  q[i] = it;
  while (i > 0) {
    int64_t parent = (i - 1) / 2;
    if (!orc_pq_less(&q[i], &q[parent])) break;
    orc_pq_item t = q[i];
    q[i] = q[parent];
    q[parent] = t;
    i = parent;
  }
}

static orc_pq_item orc_pq_pop(orc_pq_item* q, int64_t* n) {
  orc_pq_item top = q[0];
  q[0] = q[--(*n)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *n && orc_pq_less(&q[l], &q[m])) m = l;
    if (r < *n && orc_pq_less(&q[r], &q[m])) m = r;
    if (m == i) break;
    orc_pq_item t = q[i];
    q[i] = q[m];
    q[m] = t;
    i = m;
  }
  return top;
}

/* The flood on values held as doubles; `f32` rounds every filled value to
 * float and steps by float ulps (the FP32 form). */
static int orc_fill_impl(int nx, int ny, const double* h, double* w, int f32) {
  int64_t n = (int64_t)nx * ny;
  uint8_t* closed = (uint8_t*)calloc((size_t)n, 1);
  orc_pq_item* q = (orc_pq_item*)malloc(sizeof(orc_pq_item) * (size_t)(n > 0 ? n : 1));
  if (!closed || !q) {
    free(closed);
    free(q);
    return -1;
  }
  int64_t qn = 0;
  for (int y = 0; y < ny; ++y) {
    for (int x = 0; x < nx; ++x) {
      if (!orc_on_perimeter(nx, ny, x, y)) continue;
      int64_t c = (int64_t)y * nx + x;
      w[c] = h[c];
      closed[c] = 1;
      orc_pq_item it = {w[c], c};
      orc_pq_push(q, &qn, it);
    }
  }
  while (qn > 0) {
    orc_pq_item it = orc_pq_pop(q, &qn);
    int64_t c = it.c;
    int x = (int)(c % nx), y = (int)(c / nx);
    double up = f32 ? (double)nextafterf((float)w[c], INFINITY) : nextafter(w[c], INFINITY);
    for (int k = 0; k < 8; ++k) {
      int xn = x + ORC_DX[k], yn = y + ORC_DY[k];
      if (xn < 0 || yn < 0 || xn >= nx || yn >= ny) continue;
      int64_t nb = (int64_t)yn * nx + xn;
      if (closed[nb]) continue;
      closed[nb] = 1;
      w[nb] = h[nb] > up ? h[nb] : up;
      orc_pq_item nt = {w[nb], nb};
      orc_pq_push(q, &qn, nt);
    }
  }
  free(closed);
  free(q);
  return 0;
}

int orc_fill_eps(int nx, int ny, const double* h, double* w) {
  return orc_fill_impl(nx, ny, h, w, 0);
}

int orc_fill_eps_f32(int nx, int ny, const float* h, float* w) {
  int64_t n = (int64_t)nx * ny;
  double* hd = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* wd = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!hd || !wd) {
    free(hd);
    free(wd);
    return -1;
  }
  for (int64_t c = 0; c < n; ++c) hd[c] = (double)h[c];
  int rc = orc_fill_impl(nx, ny, hd, wd, 1);
  for (int64_t c = 0; c < n && rc == 0; ++c) w[c] = (float)wd[c];
  free(hd);
  free(wd);
  return rc;
}

/* ---- Rinse, Repeat -------------------------------------------------------- */

int orc_run(int nx, int ny, double* h, int nsteps, const orc_params* p,
            const int32_t* frozen_rec, int64_t* nlevels_out) {
  int64_t n = (int64_t)nx * ny;
  int32_t* rec = (int32_t*)malloc(sizeof(int32_t) * n);
  int32_t* dnum = (int32_t*)malloc(sizeof(int32_t) * n);
  int32_t* donor = (int32_t*)malloc(sizeof(int32_t) * 8 * n);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * n);
  int32_t* depth = (int32_t*)malloc(sizeof(int32_t) * n);
  int64_t* levels = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * n);
  int rc = 0;
  if (!rec || !dnum || !donor || !queue || !depth || !levels || !cnt) {
    rc = -1;
    goto done;
  }
  for (int s = 0; s < nsteps; ++s) {
    if (frozen_rec)
      memcpy(rec, frozen_rec, sizeof(int32_t) * n);
    else
      orc_receivers(nx, ny, h, rec);
    orc_donors_grid(nx, ny, rec, dnum, donor);
    int64_t L = orc_queue(n, rec, 8, dnum, donor, queue, levels, depth);
    orc_accumulate(n, queue, levels, L, 8, dnum, donor, cnt);
    orc_uplift(nx, ny, h, p);
    orc_erode(nx, ny, h, rec, queue, levels, L, cnt, p);
    if (nlevels_out) nlevels_out[s] = L;
  }
done:
  free(rec);
  free(dnum);
  free(donor);
  free(queue);
  free(depth);
  free(levels);
  free(cnt);
  return rc;
}

/* ---- Adjoint and tangent-linear of one n-hat = 1 step ---------------------- */

/* F and dF/dK = dt*A^m/d of the eroding cell c. */
static void orc_F(int nx, int32_t c, int32_t r, int64_t count, const orc_params* p,
                  double* F, double* G) {
  double A = (double)count * p->area_scale;
  double d = orc_dist(nx, c, r, p->dx);
  *F = p->K * p->dt * pow(A, p->m) / d;
  *G = p->dt * pow(A, p->m) / d;
}

void orc_tangent_step(int nx, int ny, const double* h_next, const int32_t* rec,
                      const int32_t* queue, const int64_t* levels, int64_t nlevels,
                      const int64_t* cnt, const orc_params* p, const double* dh,
                      const double* dU, double dK, double* dh_next) {
  /* Level 0: perimeter cells keep h; interior pits take uplift only. */
  for (int64_t i = levels[0]; i < levels[1]; ++i) {
    int32_t c = queue[i];
    int x = c % nx, y = c / nx;
    if (orc_on_perimeter(nx, ny, x, y))
      dh_next[c] = dh[c];
    else
      dh_next[c] = dh[c] + p->dt * dU[c];
  }
  /* Levels 1.., receivers first:
   * (1+F) dh'_c = dh_c + dt dU_c + F dh'_r + dF (h'_r - h'_c),  dF = G dK. */
  for (int64_t l = 1; l < nlevels; ++l) {
    for (int64_t i = levels[l]; i < levels[l + 1]; ++i) {
      int32_t c = queue[i];
      int32_t r = rec[c];
      double F, G;
      orc_F(nx, c, r, cnt[c], p, &F, &G);
      double num = dh[c] + p->dt * dU[c] + F * dh_next[r] + G * dK * (h_next[r] - h_next[c]);
      dh_next[c] = num / (1.0 + F);
    }
  }
}

void orc_adjoint_step(int nx, int ny, const double* h_next, const int32_t* rec,
                      const int32_t* queue, const int64_t* levels, int64_t nlevels,
                      const int64_t* cnt, const orc_params* p, const double* lam,
                      double* lam_prev, double* dLdU, double* dLdK) {
  int64_t n = (int64_t)nx * ny;
  double* mu = (double*)malloc(sizeof(double) * n);
  if (!mu) return;
  for (int64_t c = 0; c < n; ++c) mu[c] = lam[c];
  /* Transpose of the receivers-first sweep: donors first (levels high to 1),
   * each eroding cell passing mu_c * F_c/(1+F_c) to its receiver. */
  for (int64_t l = nlevels - 1; l >= 1; --l) {
    for (int64_t i = levels[l]; i < levels[l + 1]; ++i) {
      int32_t c = queue[i];
      int32_t r = rec[c];
      double F, G;
      orc_F(nx, c, r, cnt[c], p, &F, &G);
      mu[r] = mu[r] + mu[c] * (F / (1.0 + F));
    }
  }
  double gK = 0.0;
  for (int64_t l = 1; l < nlevels; ++l) {
    for (int64_t i = levels[l]; i < levels[l + 1]; ++i) {
      int32_t c = queue[i];
      int32_t r = rec[c];
      double F, G;
      orc_F(nx, c, r, cnt[c], p, &F, &G);
      lam_prev[c] = mu[c] / (1.0 + F);
      dLdU[c] = dLdU[c] + p->dt * mu[c] / (1.0 + F);
      gK = gK + mu[c] * G * (h_next[r] - h_next[c]) / (1.0 + F);
    }
  }
  for (int64_t i = levels[0]; i < levels[1]; ++i) {
    int32_t c = queue[i];
    int x = c % nx, y = c / nx;
    lam_prev[c] = mu[c];
    if (!orc_on_perimeter(nx, ny, x, y)) dLdU[c] = dLdU[c] + p->dt * mu[c];
  }
  *dLdK = *dLdK + gK;
  free(mu);
}
