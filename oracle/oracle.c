/*
 * FP64 CPU oracle for run-time loop-chain tiling (Reguly, Mudalige, Giles,
 * "Loop Tiling in Large-Scale Stencil Codes at Run-time with OPS").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity reference for the CUDA
 * library: only the tests, the package smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header or table with the
 * library; it decodes the loop-chain interchange format (register IR,
 * argument lists, stencils) with its own definitions.
 *
 * What it computes:
 *  - ora_run_loops: the plain untiled program-order execution of a chain of
 *    parallel loops, in FP64 or (f32) in FP32.  A parallel loop's result must not depend on the order
 *    of its points (Sec. 3), and tiling only reorders such work (Sec. 4.B,
 *    Algorithm 2), so the untiled result is what every tiled schedule must
 *    reproduce.  Each point evaluates the IR in its fixed statement and term
 *    order with explicit fma; the build uses -ffp-contract=off.
 *  - reductions: sums are exactly rounded (Shewchuk's exact partials, the
 *    method behind Python's math.fsum); min/max are exact.
 *  - ora_cg64 / ora_cg_refine: textbook conjugate gradients (Hestenes and
 *    Stiefel) on the 5-point heat-conduction operator, in FP64, and an FP32
 *    inner CG inside FP64 iterative refinement; dots are exact sums of the
 *    rounded products.
 *
 * Every grid access is bounds-checked against the dat's allocation; a
 * violation returns an error instead of reading outside the array.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- interchange-format numbers, decoded independently of the library ---- */
enum { I_LD = 1, I_CST, I_ADD, I_SUB, I_MUL, I_FMA, I_DIV, I_MIN, I_MAX, I_SGT,
       I_WSUM, I_WACC, I_POLY, I_ST, I_RED };
enum { K_DAT = 0, K_SCALAR = 1, K_RED = 2 };
enum { A_READ = 0, A_WRITE = 1, A_RW = 2, A_INC = 3 };
enum { R_SUM = 0, R_MIN = 1, R_MAX = 2 };
#define NREG 8

/* ---------------------------------------------------------------------------
 * Exactly rounded summation (J. R. Shewchuk, "Adaptive precision
 * floating-point arithmetic and fast robust geometric predicates", 1997):
 * keep the running sum as non-overlapping partials of increasing magnitude,
 * each addition exact; round once at the end, half-way cases to even.
 * ------------------------------------------------------------------------- */
typedef struct { double* p; int n, cap; } xsum;

static void xs_init(xsum* s) { s->p = NULL; s->n = 0; s->cap = 0; }
static void xs_free(xsum* s) { free(s->p); s->p = NULL; s->n = s->cap = 0; }

static void xs_add(xsum* s, double x) {
  int i = 0;
  for (int j = 0; j < s->n; ++j) {
    double y = s->p[j];
    if (fabs(x) < fabs(y)) { double t = x; x = y; y = t; }
    double hi = x + y;
    double lo = y - (hi - x);
    if (lo != 0.0) s->p[i++] = lo;
    x = hi;
  }
  if (i >= s->cap) {
    int nc = s->cap ? 2 * s->cap : 16;
    s->p = (double*)realloc(s->p, sizeof(double) * (size_t)nc);
    s->cap = nc;
  }
  s->p[i++] = x;
  s->n = i;
}

static double xs_round(const xsum* s) {
  int n = s->n;
  if (n == 0) return 0.0;
  double hi = s->p[--n], lo = 0.0;
  while (n > 0) {
    double x = hi, y = s->p[--n];
    hi = x + y;
    double yr = hi - x;
    lo = y - yr;
    if (lo != 0.0) break;
  }
  /* the partials below lo decide a tie: push towards them if same sign */
  if (n > 0 && ((lo < 0.0 && s->p[n - 1] < 0.0) || (lo > 0.0 && s->p[n - 1] > 0.0))) {
    double y = lo * 2.0, x = hi + y, yr = x - hi;
    if (y == yr) hi = x;
  }
  return hi;
}

double ora_fsum(const double* x, int64_t n) {
  xsum s; xs_init(&s);
  for (int64_t i = 0; i < n; ++i) xs_add(&s, x[i]);
  double r = xs_round(&s);
  xs_free(&s);
  return r;
}

/* exactly rounded dot product of the rounded products fl(x_i * y_i) */
static double xdot(const double* x, const double* y, int64_t n) {
  xsum s; xs_init(&s);
  for (int64_t i = 0; i < n; ++i) xs_add(&s, x[i] * y[i]);
  double r = xs_round(&s);
  xs_free(&s);
  return r;
}

/* exactly rounded dot of FP32 vectors: the products of two floats are exact
 * in FP64, so this is the exactly rounded value of the exact dot product */
static double xdot32(const float* x, const float* y, int64_t n) {
  xsum s; xs_init(&s);
  for (int64_t i = 0; i < n; ++i) xs_add(&s, (double)x[i] * (double)y[i]);
  double r = xs_round(&s);
  xs_free(&s);
  return r;
}

/* ---------------------------------------------------------------------------
 * Untiled program-order interpreter
 * ------------------------------------------------------------------------- */
typedef struct {
  int ndats;
  double** dat;           /* dense, x fastest, allocated box incl. halos (float* when f32) */
  const int* ext;         /* 3 per dat: allocated extents ex, ey, ez */
  const int* dm;          /* 3 per dat: index of grid point 0 inside the allocation */
  const int* st_npts;
  const int* st_start;    /* first point of each stencil in st_off */
  const int* st_off;      /* 3 ints per stencil point */
  int nred;
  const int* red_op;
  int f32;                /* 1: FP32 dats and FP32 arithmetic (IEEE single, explicit fmaf) */
} env_t;

typedef struct {
  const int* rng;         /* 6 ints: x0 x1 y0 y1 z0 z1 */
  int nargs;
  const int* args;        /* 4 ints per arg: kind handle stencil access */
  int nins;
  const int* ins;         /* 6 ints per instruction */
  const double* K;
  int nK;
} loop_t;

typedef struct {
  int err;
  char msg[256];
} status_t;

static void fail(status_t* st, const char* fmt, long a, long b, long c) {
#pragma omp critical(oracle_fail)
  {
    if (!st->err) {
      st->err = 1;
      snprintf(st->msg, sizeof st->msg, fmt, a, b, c);
    }
  }
}

/* address of dat element at grid point (x, y, z), or NULL outside the allocation */
static double* at(const env_t* E, int dat, long x, long y, long z) {
  const int* e = E->ext + 3 * dat;
  const int* m = E->dm + 3 * dat;
  long ix = x + m[0], iy = y + m[1], iz = z + m[2];
  if (ix < 0 || iy < 0 || iz < 0 || ix >= e[0] || iy >= e[1] || iz >= e[2]) return NULL;
  return E->dat[dat] + ix + (long)e[0] * (iy + (long)e[1] * iz);
}

typedef struct {
  xsum* sums;     /* per reduction handle */
  double* mm;     /* running min / max per reduction handle */
  int* touched;
} redacc_t;

/* value of a stencil point of a DAT argument */
static int fetch(const env_t* E, const loop_t* L, int a, int p, long x, long y, long z,
                 double* out, status_t* st) {
  const int* ar = L->args + 4 * a;
  if (ar[0] != K_DAT) { fail(st, "LD of a non-dat argument %ld", a, 0, 0); return 0; }
  int s = ar[2];
  if (p < 0 || p >= E->st_npts[s]) { fail(st, "stencil point %ld out of range for arg %ld", p, a, 0); return 0; }
  const int* o = E->st_off + 3 * (E->st_start[s] + p);
  double* q = at(E, ar[1], x + o[0], y + o[1], z + o[2]);
  if (!q) { fail(st, "out-of-allocation read at (%ld,%ld,%ld)", x + o[0], y + o[1], z + o[2]); return 0; }
  *out = *q;
  return 1;
}

static void run_point(const env_t* E, const loop_t* L, const double* scal, long x, long y, long z,
                      redacc_t* acc, status_t* st) {
  double r[NREG];
  for (int i = 0; i < NREG; ++i) r[i] = 0.0;
  for (int pc = 0; pc < L->nins; ++pc) {
    const int* I = L->ins + 6 * pc;
    int op = I[0], d = I[1], a = I[2], b = I[3], c = I[4], e = I[5];
    double v;
    switch (op) {
      case I_LD:
        if (L->args[4 * a] == K_SCALAR) { r[d] = scal[L->args[4 * a + 1]]; break; }
        if (!fetch(E, L, a, b, x, y, z, &v, st)) return;
        r[d] = v;
        break;
      case I_CST: r[d] = L->K[a]; break;
      case I_ADD: r[d] = r[a] + r[b]; break;
      case I_SUB: r[d] = r[a] - r[b]; break;
      case I_MUL: r[d] = r[a] * r[b]; break;
      case I_FMA: r[d] = fma(r[a], r[b], r[c]); break;
      case I_DIV: r[d] = r[a] / r[b]; break;
      case I_MIN: r[d] = (r[b] < r[a]) ? r[b] : r[a]; break;
      case I_MAX: r[d] = (r[b] > r[a]) ? r[b] : r[a]; break;
      case I_SGT: r[d] = (r[a] > r[b]) ? r[c] : r[e]; break;
      case I_WSUM:
      case I_WACC: {
        int s = L->args[4 * a + 2];
        int np = E->st_npts[s];
        double t = r[d];
        for (int p = 0; p < np; ++p) {
          if (!fetch(E, L, a, p, x, y, z, &v, st)) return;
          if (op == I_WSUM && p == 0) t = L->K[b] * v;
          else t = fma(L->K[b + p], v, t);
        }
        r[d] = t;
        break;
      }
      case I_POLY: {
        double t = L->K[b + c];
        for (int i = c - 1; i >= 0; --i) t = fma(t, r[a], L->K[b + i]);
        r[d] = t;
        break;
      }
      case I_ST: {
        const int* ar = L->args + 4 * d;
        double* q = at(E, ar[1], x, y, z);
        if (!q) { fail(st, "out-of-allocation write at (%ld,%ld,%ld)", x, y, z); return; }
        if (ar[3] == A_INC) *q = *q + r[a];
        else *q = r[a];
        break;
      }
      case I_RED: {
        int h = L->args[4 * d + 1];
        int rop = E->red_op[h];
        acc->touched[h] = 1;
        if (rop == R_SUM) xs_add(&acc->sums[h], r[a]);
        else if (rop == R_MIN) acc->mm[h] = (r[a] < acc->mm[h]) ? r[a] : acc->mm[h];
        else acc->mm[h] = (r[a] > acc->mm[h]) ? r[a] : acc->mm[h];
        break;
      }
      default:
        fail(st, "bad opcode %ld at %ld", op, pc, 0);
        return;
    }
  }
}

/* ---- FP32: the same interpreter on float dats, every operation an IEEE
 * single operation (C float arithmetic, fmaf), constants and scalars rounded
 * to float on load; reductions take the float values exactly ---- */
static float* at32(const env_t* E, int dat, long x, long y, long z) {
  const int* e = E->ext + 3 * dat;
  const int* m = E->dm + 3 * dat;
  long ix = x + m[0], iy = y + m[1], iz = z + m[2];
  if (ix < 0 || iy < 0 || iz < 0 || ix >= e[0] || iy >= e[1] || iz >= e[2]) return NULL;
  return ((float*)E->dat[dat]) + ix + (long)e[0] * (iy + (long)e[1] * iz);
}

static int fetch32(const env_t* E, const loop_t* L, int a, int p, long x, long y, long z,
                   float* out, status_t* st) {
  const int* ar = L->args + 4 * a;
  if (ar[0] != K_DAT) { fail(st, "LD of a non-dat argument %ld", a, 0, 0); return 0; }
  int s = ar[2];
  if (p < 0 || p >= E->st_npts[s]) { fail(st, "stencil point %ld out of range for arg %ld", p, a, 0); return 0; }
  const int* o = E->st_off + 3 * (E->st_start[s] + p);
  float* q = at32(E, ar[1], x + o[0], y + o[1], z + o[2]);
  if (!q) { fail(st, "out-of-allocation read at (%ld,%ld,%ld)", x + o[0], y + o[1], z + o[2]); return 0; }
  *out = *q;
  return 1;
}

static void run_point32(const env_t* E, const loop_t* L, const double* scal, long x, long y, long z,
                        redacc_t* acc, status_t* st) {
  float r[NREG];
  for (int i = 0; i < NREG; ++i) r[i] = 0.0f;
  for (int pc = 0; pc < L->nins; ++pc) {
    const int* I = L->ins + 6 * pc;
    int op = I[0], d = I[1], a = I[2], b = I[3], c = I[4], e = I[5];
    float v;
    switch (op) {
      case I_LD:
        if (L->args[4 * a] == K_SCALAR) { r[d] = (float)scal[L->args[4 * a + 1]]; break; }
        if (!fetch32(E, L, a, b, x, y, z, &v, st)) return;
        r[d] = v;
        break;
      case I_CST: r[d] = (float)L->K[a]; break;
      case I_ADD: r[d] = r[a] + r[b]; break;
      case I_SUB: r[d] = r[a] - r[b]; break;
      case I_MUL: r[d] = r[a] * r[b]; break;
      case I_FMA: r[d] = fmaf(r[a], r[b], r[c]); break;
      case I_DIV: r[d] = r[a] / r[b]; break;
      case I_MIN: r[d] = (r[b] < r[a]) ? r[b] : r[a]; break;
      case I_MAX: r[d] = (r[b] > r[a]) ? r[b] : r[a]; break;
      case I_SGT: r[d] = (r[a] > r[b]) ? r[c] : r[e]; break;
      case I_WSUM:
      case I_WACC: {
        int s = L->args[4 * a + 2];
        int np = E->st_npts[s];
        float t = r[d];
        for (int p = 0; p < np; ++p) {
          if (!fetch32(E, L, a, p, x, y, z, &v, st)) return;
          if (op == I_WSUM && p == 0) t = (float)L->K[b] * v;
          else t = fmaf((float)L->K[b + p], v, t);
        }
        r[d] = t;
        break;
      }
      case I_POLY: {
        float t = (float)L->K[b + c];
        for (int i = c - 1; i >= 0; --i) t = fmaf(t, r[a], (float)L->K[b + i]);
        r[d] = t;
        break;
      }
      case I_ST: {
        const int* ar = L->args + 4 * d;
        float* q = at32(E, ar[1], x, y, z);
        if (!q) { fail(st, "out-of-allocation write at (%ld,%ld,%ld)", x, y, z); return; }
        if (ar[3] == A_INC) *q = *q + r[a];
        else *q = r[a];
        break;
      }
      case I_RED: {
        int h = L->args[4 * d + 1];
        int rop = E->red_op[h];
        double w = (double)r[a];
        acc->touched[h] = 1;
        if (rop == R_SUM) xs_add(&acc->sums[h], w);
        else if (rop == R_MIN) acc->mm[h] = (w < acc->mm[h]) ? w : acc->mm[h];
        else acc->mm[h] = (w > acc->mm[h]) ? w : acc->mm[h];
        break;
      }
      default:
        fail(st, "bad opcode %ld at %ld", op, pc, 0);
        return;
    }
  }
}

/* reduction state: an exact sum per SUM handle, a running value per MIN/MAX */
typedef struct { xsum* sums; double* mm; } redstate_t;

static double red_value(const env_t* E, const redstate_t* R, int h) {
  return E->red_op[h] == R_SUM ? xs_round(&R->sums[h]) : R->mm[h];
}

static void run_loop(const env_t* E, const loop_t* L, redstate_t* RS, int nthreads, status_t* st) {
  long x0 = L->rng[0], x1 = L->rng[1], y0 = L->rng[2], y1 = L->rng[3], z0 = L->rng[4], z1 = L->rng[5];
  if (x1 <= x0 || y1 <= y0 || z1 <= z0) return;
  /* scalar arguments see the reduction values from before this loop */
  double* scal = (double*)calloc((size_t)(E->nred > 0 ? E->nred : 1), sizeof(double));
  for (int h = 0; h < E->nred; ++h) scal[h] = red_value(E, RS, h);
  long nz = z1 - z0, ny = y1 - y0;
  long nouter = nz * ny;
#ifdef _OPENMP
  int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  int nt = 1;
  (void)nthreads;
#endif
  redacc_t* accs = (redacc_t*)calloc((size_t)nt, sizeof(redacc_t));
  for (int t = 0; t < nt; ++t) {
    accs[t].sums = (xsum*)calloc((size_t)(E->nred + 1), sizeof(xsum));
    accs[t].mm = (double*)calloc((size_t)(E->nred + 1), sizeof(double));
    accs[t].touched = (int*)calloc((size_t)(E->nred + 1), sizeof(int));
    for (int h = 0; h < E->nred; ++h) {
      xs_init(&accs[t].sums[h]);
      accs[t].mm[h] = E->red_op[h] == R_MIN ? INFINITY : -INFINITY;
    }
  }
#pragma omp parallel for schedule(static) num_threads(nt)
  for (long o = 0; o < nouter; ++o) {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    long z = z0 + o / ny, y = y0 + o % ny;
    for (long x = x0; x < x1; ++x) {
      if (st->err) break;
      if (E->f32)
        run_point32(E, L, scal, x, y, z, &accs[tid], st);
      else
        run_point(E, L, scal, x, y, z, &accs[tid], st);
    }
  }
  /* fold per-thread reduction state into the handles (exact for sums) */
  for (int t = 0; t < nt; ++t) {
    for (int h = 0; h < E->nred; ++h) {
      if (accs[t].touched[h]) {
        if (E->red_op[h] == R_SUM) {
          for (int i = 0; i < accs[t].sums[h].n; ++i) xs_add(&RS->sums[h], accs[t].sums[h].p[i]);
        } else if (E->red_op[h] == R_MIN) {
          RS->mm[h] = (accs[t].mm[h] < RS->mm[h]) ? accs[t].mm[h] : RS->mm[h];
        } else {
          RS->mm[h] = (accs[t].mm[h] > RS->mm[h]) ? accs[t].mm[h] : RS->mm[h];
        }
      }
      xs_free(&accs[t].sums[h]);
    }
    free(accs[t].sums);
    free(accs[t].mm);
    free(accs[t].touched);
  }
  free(accs);
  free(scal);
}

/*
 * Run `nloops` loops in program order over the given dats (modified in
 * place; float arrays and FP32 arithmetic when f32 != 0).  red_val[h] holds each reduction's value on entry (the identity
 * after a host read) and its exactly rounded / exact value on return.
 * Returns 0, or 1 with a message in errbuf (>= 256 bytes).
 */
int ora_run_loops(int ndats, double** dat, const int* ext, const int* dm,
                  const int* st_npts, const int* st_start, const int* st_off,
                  int nred, const int* red_op, double* red_val,
                  int nloops, const int* loop_rng, const int* loop_nargs, const int* loop_arg0,
                  const int* args, const int* loop_nins, const int* loop_ins0, const int* ins,
                  const int* loop_k0, const int* loop_nk, const double* K,
                  int nthreads, int f32, char* errbuf) {
  env_t E = {ndats, dat, ext, dm, st_npts, st_start, st_off, nred, red_op, f32};
  status_t st;
  st.err = 0;
  st.msg[0] = 0;
  redstate_t RS;
  RS.sums = (xsum*)calloc((size_t)(nred + 1), sizeof(xsum));
  RS.mm = (double*)calloc((size_t)(nred + 1), sizeof(double));
  for (int h = 0; h < nred; ++h) {
    xs_init(&RS.sums[h]);
    if (red_op[h] == R_SUM) xs_add(&RS.sums[h], red_val[h]);
    else RS.mm[h] = red_val[h];
  }
  for (int l = 0; l < nloops && !st.err; ++l) {
    loop_t L = {loop_rng + 6 * l, loop_nargs[l], args + 4 * loop_arg0[l], loop_nins[l],
                ins + 6 * loop_ins0[l], K + loop_k0[l], loop_nk[l]};
    run_loop(&E, &L, &RS, nthreads, &st);
    if (st.err) {
      char tmp[256];
      snprintf(tmp, sizeof tmp, "loop %d: %s", l, st.msg);
      memcpy(st.msg, tmp, sizeof tmp);
    }
  }
  for (int h = 0; h < nred; ++h) {
    red_val[h] = red_value(&E, &RS, h);
    xs_free(&RS.sums[h]);
  }
  free(RS.sums);
  free(RS.mm);
  if (errbuf) snprintf(errbuf, 256, "%s", st.msg);
  return st.err;
}

/* ---------------------------------------------------------------------------
 * Heat-conduction operator on an n x n cell grid (x fastest):
 *   (A u)_c = u_c + sum over the 4 faces f of c of k_f (u_c - u_nb),
 * k_f the harmonic mean 2 ka kb / (ka + kb) of the two cells' conductivity;
 * a boundary face takes the cell's own conductivity and u_nb = 0 outside.
 * Evaluated as d_c u_c - kW uW - kE uE - kS uS - kN uN with
 * d_c = (((1 + kW) + kE) + kS) + kN, the products applied by fma in the
 * order W, E, S, N.
 * kx: n rows of n+1 faces (face i sits between cells i-1 and i);
 * ky: n+1 rows of n faces (face row j sits between cell rows j-1 and j).
 * ------------------------------------------------------------------------- */
static double hmean(double a, double b) { return (2.0 * a * b) / (a + b); }

void ora_faces(int n, const double* kappa, double* kx, double* ky, double* diag) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= n; ++i) {
      double k;
      if (i == 0) k = kappa[(long)j * n];
      else if (i == n) k = kappa[(long)j * n + n - 1];
      else k = hmean(kappa[(long)j * n + i - 1], kappa[(long)j * n + i]);
      kx[(long)j * (n + 1) + i] = k;
    }
  for (int j = 0; j <= n; ++j)
    for (int i = 0; i < n; ++i) {
      double k;
      if (j == 0) k = kappa[i];
      else if (j == n) k = kappa[(long)(n - 1) * n + i];
      else k = hmean(kappa[(long)(j - 1) * n + i], kappa[(long)j * n + i]);
      ky[(long)j * n + i] = k;
    }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double d = 1.0 + kx[(long)j * (n + 1) + i];
      d = d + kx[(long)j * (n + 1) + i + 1];
      d = d + ky[(long)j * n + i];
      d = d + ky[(long)(j + 1) * n + i];
      diag[(long)j * n + i] = d;
    }
}

void ora_matvec(int n, const double* kx, const double* ky, const double* diag, const double* u, double* w) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      long c = (long)j * n + i;
      double uW = i > 0 ? u[c - 1] : 0.0;
      double uE = i < n - 1 ? u[c + 1] : 0.0;
      double uS = j > 0 ? u[c - n] : 0.0;
      double uN = j < n - 1 ? u[c + n] : 0.0;
      double t = diag[c] * u[c];
      t = fma(-kx[(long)j * (n + 1) + i], uW, t);
      t = fma(-kx[(long)j * (n + 1) + i + 1], uE, t);
      t = fma(-ky[(long)j * n + i], uS, t);
      t = fma(-ky[(long)(j + 1) * n + i], uN, t);
      w[c] = t;
    }
}

/* FP32 operator: coefficients rounded to float, same term order with fmaf */
void ora_matvec32(int n, const float* kx, const float* ky, const float* diag, const float* u, float* w) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      long c = (long)j * n + i;
      float uW = i > 0 ? u[c - 1] : 0.0f;
      float uE = i < n - 1 ? u[c + 1] : 0.0f;
      float uS = j > 0 ? u[c - n] : 0.0f;
      float uN = j < n - 1 ? u[c + n] : 0.0f;
      float t = diag[c] * u[c];
      t = fmaf(-kx[(long)j * (n + 1) + i], uW, t);
      t = fmaf(-kx[(long)j * (n + 1) + i + 1], uE, t);
      t = fmaf(-ky[(long)j * n + i], uS, t);
      t = fmaf(-ky[(long)(j + 1) * n + i], uN, t);
      w[c] = t;
    }
}

/*
 * FP64 conjugate gradients from x = 0 until ||r||_2 <= tol ||b||_2 (r the
 * recursively updated residual) or maxit iterations.  Returns the number of
 * iterations; *relres receives ||r||/||b|| of the recursive residual.
 */
int ora_cg64(int n, const double* kappa, const double* b, double tol, int maxit, double* x, double* relres) {
  long N = (long)n * n;
  double* kx = malloc(sizeof(double) * (size_t)(n * (long)(n + 1)));
  double* ky = malloc(sizeof(double) * (size_t)(n * (long)(n + 1)));
  double* dg = malloc(sizeof(double) * (size_t)N);
  double* r = malloc(sizeof(double) * (size_t)N);
  double* p = malloc(sizeof(double) * (size_t)N);
  double* w = malloc(sizeof(double) * (size_t)N);
  ora_faces(n, kappa, kx, ky, dg);
  for (long i = 0; i < N; ++i) { x[i] = 0.0; r[i] = b[i]; p[i] = b[i]; }
  double bb = xdot(b, b, N);
  double rr = bb;
  int it = 0;
  double nb = sqrt(bb);
  while (it < maxit && sqrt(rr) > tol * nb) {
    ora_matvec(n, kx, ky, dg, p, w);
    double pw = xdot(p, w, N);
    double alpha = rr / pw;
    for (long i = 0; i < N; ++i) {
      x[i] = fma(alpha, p[i], x[i]);
      r[i] = fma(-alpha, w[i], r[i]);
    }
    double rr1 = xdot(r, r, N);
    ++it;
    double beta = rr1 / rr;
    rr = rr1;
    if (sqrt(rr) <= tol * nb) break;
    for (long i = 0; i < N; ++i) p[i] = fma(beta, p[i], r[i]);
  }
  *relres = sqrt(rr) / nb;
  free(kx); free(ky); free(dg); free(r); free(p); free(w);
  return it;
}

/* ||b - A x||_2 / ||b||_2 in FP64 with exact norms */
double ora_relres(int n, const double* kappa, const double* b, const double* x) {
  long N = (long)n * n;
  double* kx = malloc(sizeof(double) * (size_t)(n * (long)(n + 1)));
  double* ky = malloc(sizeof(double) * (size_t)(n * (long)(n + 1)));
  double* dg = malloc(sizeof(double) * (size_t)N);
  double* w = malloc(sizeof(double) * (size_t)N);
  ora_faces(n, kappa, kx, ky, dg);
  ora_matvec(n, kx, ky, dg, x, w);
  for (long i = 0; i < N; ++i) w[i] = b[i] - w[i];
  double rr = xdot(w, w, N), bb = xdot(b, b, N);
  free(kx); free(ky); free(dg); free(w);
  return sqrt(rr) / sqrt(bb);
}

/*
 * Mixed-precision iterative refinement: r = b - A x in FP64; stop when
 * ||r|| <= tol ||b||; else solve A d = r / ||r|| with FP32 CG (FP32 vectors
 * and operator, FP64 dot accumulation and scalars) to relative residual
 * inner_tol, and update x = fma(||r||, d, x) in FP64.
 * Returns total inner iterations; *outer the number of corrections.
 */
int ora_cg_refine(int n, const double* kappa, const double* b, double tol, double inner_tol,
                  int maxit, int maxouter, double* x, double* relres, int* outer) {
  long N = (long)n * n;
  double* kx = malloc(sizeof(double) * (size_t)(n * (long)(n + 1)));
  double* ky = malloc(sizeof(double) * (size_t)(n * (long)(n + 1)));
  double* dg = malloc(sizeof(double) * (size_t)N);
  double* r = malloc(sizeof(double) * (size_t)N);
  float* kxf = malloc(sizeof(float) * (size_t)(n * (long)(n + 1)));
  float* kyf = malloc(sizeof(float) * (size_t)(n * (long)(n + 1)));
  float* dgf = malloc(sizeof(float) * (size_t)N);
  float* rf = malloc(sizeof(float) * (size_t)N);
  float* pf = malloc(sizeof(float) * (size_t)N);
  float* wf = malloc(sizeof(float) * (size_t)N);
  float* df = malloc(sizeof(float) * (size_t)N);
  ora_faces(n, kappa, kx, ky, dg);
  for (long i = 0; i < n * (long)(n + 1); ++i) { kxf[i] = (float)kx[i]; kyf[i] = (float)ky[i]; }
  for (long i = 0; i < N; ++i) { dgf[i] = (float)dg[i]; x[i] = 0.0; }
  double nb = sqrt(xdot(b, b, N));
  int total = 0, o = 0;
  double rel = 1.0;
  for (;;) {
    ora_matvec(n, kx, ky, dg, x, r);
    for (long i = 0; i < N; ++i) r[i] = b[i] - r[i];
    double nr = sqrt(xdot(r, r, N));
    rel = nr / nb;
    if (rel <= tol || o >= maxouter || total >= maxit) break;
    double inv = 1.0 / nr;
    for (long i = 0; i < N; ++i) { rf[i] = (float)(r[i] * inv); pf[i] = rf[i]; df[i] = 0.0f; }
    double rho = xdot32(rf, rf, N);
    double rho0 = rho;
    int it = 0;
    while (total < maxit) {
      ora_matvec32(n, kxf, kyf, dgf, pf, wf);
      double pw = xdot32(pf, wf, N);
      double alpha = rho / pw;
      float af = (float)alpha;
      for (long i = 0; i < N; ++i) {
        df[i] = fmaf(af, pf[i], df[i]);
        rf[i] = fmaf(-af, wf[i], rf[i]);
      }
      double rho1 = xdot32(rf, rf, N);
      ++it;
      ++total;
      if (sqrt(rho1) <= inner_tol * sqrt(rho0)) break;
      float bf = (float)(rho1 / rho);
      rho = rho1;
      for (long i = 0; i < N; ++i) pf[i] = fmaf(bf, pf[i], rf[i]);
    }
    for (long i = 0; i < N; ++i) x[i] = fma(nr, (double)df[i], x[i]);
    ++o;
  }
  *relres = rel;
  *outer = o;
  free(kx); free(ky); free(dg); free(r); free(kxf); free(kyf); free(dgf);
  free(rf); free(pf); free(wf); free(df);
  return total;
}
