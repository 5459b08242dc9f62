/*
 * hygt_oracle.c -- plain, slow CPU oracle for the Hypercube-Givens Transform
 * (HyGT) of Said et al., "Highly Efficient Non-Separable Transforms for Next
 * Generation Video Coding".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library: every table below is recomputed here from its definition.
 *
 * What it computes, in the paper's order and notation:
 *
 *   - Givens rotation G(m,n,theta) (Sec. IV): on the pair of entries (m,n) it
 *     maps (a,b) to (cos*a + sin*b, -sin*a + cos*b); every other entry is
 *     kept.
 *   - Parallel-Givens pass (Sec. IV, pair-cover equation and the
 *     parallel-Givens product): N/2 disjoint rotations that cover 0..N-1.
 *   - HyGT round (Sec. IV, Fig. 3 and Fig. 4): log2(N) passes; pass p pairs
 *     every index m whose bit p is clear with n = m + 2^p (the edges of the
 *     log2(N)-dimensional hypercube along dimension p).  Within pass p the
 *     pairs are numbered j = 0..N/2-1 in increasing order of m, and pair j
 *     uses angle j of that pass.  Passes run p = 0,1,...,log2(N)-1.
 *   - Full HyGT (Sec. IV, Fig. 2; PMPT product Eq. 5): R rounds, each followed
 *     by an optional permutation ("sorting") slot; the first pass is applied
 *     first.  Slot r is a gather: v'[i] = v[perm[r][i]].
 *   - Inverse (Sec. III inverse product; Sec. IV inverse of the
 *     parallel-Givens matrix): the passes in reverse order, each with the
 *     negated angles, the permutations undone by a scatter.
 *   - On-the-fly parameter conversion (Sec. IV, Fig. 5): an angle index q of
 *     `angle_bits` bits (at most 8: one byte per parameter) stands for
 *     theta = 2*pi*q / 2^angle_bits; the integer multipliers are
 *     c = round(2^f cos theta), s = round(2^f sin theta) with f = `frac_bits`,
 *     rounded half away from zero.
 *   - Integer butterfly: each output of a rotation is rounded half up,
 *     y = floor((c*a + s*b + 2^(f-1)) / 2^f), computed in int64 and checked to
 *     fit in int32.  The inverse uses (c, -s) from the same table entries.
 *     The inverse output is saturated to int16.
 *   - Set index per block (Sec. II, the classification index c): 0xFFFF
 *     means "no secondary transform" (identity); any other value >= num_sets
 *     is an error and the block's output is zeroed.
 *   - Dense form T (PMPT product, Eq. 5): column i of T is the transform of
 *     the unit vector e_i, computed in FP64.
 *   - Energy-compaction loss L = (1/B) sum_b sum_{i>=K} y_{b,i}^2 and its
 *     analytic gradient, by back-propagation through stored FP64 activations.
 *
 * All functions return 0 on success or a nonzero error code (see below).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SET 4
#define OR_ERR_OVERFLOW 5

#define OR_SKIP 0xFFFFu
#define OR_MAX_N 256

static const double OR_TWO_PI = 6.283185307179586476925286766559;

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Hypercube pairing (Sec. IV, Fig. 3 / Fig. 4).                        */
/* Pair j of pass p: m is the j-th integer (in increasing order) whose  */
/* bit p is zero, i.e. j with a zero bit inserted at position p;        */
/* n = m + 2^p.                                                         */
/* ------------------------------------------------------------------ */
void oracle_pair(int p, int j, int *m, int *n) {
  int below = j & ((1 << p) - 1); /* bits of j under position p  */
  int above = j >> p;             /* bits of j from position p up */
  *m = (above << (p + 1)) | below;
  *n = *m + (1 << p);
}

/* Multiplier table of the on-the-fly conversion (Sec. IV, Fig. 5). */
int oracle_cs_table(int angle_bits, int frac_bits, int32_t *c, int32_t *s) {
  if (angle_bits < 1 || angle_bits > 8 || frac_bits < 1 || frac_bits > 14) return OR_ERR_ARG;
  int count = 1 << angle_bits;
  double scale = ldexp(1.0, frac_bits);
  for (int q = 0; q < count; ++q) {
    double theta = OR_TWO_PI * (double)q / (double)count;
    c[q] = (int32_t)lround(scale * cos(theta));
    s[q] = (int32_t)lround(scale * sin(theta));
  }
  return OR_OK;
}

/* floor(u / 2^f) for any sign of u, written as a plain division. */
static int64_t floor_div_pow2(int64_t u, int f) {
  int64_t d = (int64_t)1 << f;
  int64_t q = u / d; /* C division truncates toward zero */
  if ((u % d) != 0 && u < 0) q -= 1;
  return q;
}

static int fits_i32(int64_t u) { return u >= INT32_MIN && u <= INT32_MAX; }

static int16_t saturate_i16(int64_t v) {
  if (v > 32767) return 32767;
  if (v < -32768) return -32768;
  return (int16_t)v;
}

static int check_shape(int log2n, int rounds, int num_sets) {
  if (log2n < 1 || log2n > 8 || rounds < 1 || rounds > 16) return OR_ERR_ARG;
  if (num_sets < 1 || num_sets > 65535) return OR_ERR_ARG;
  return OR_OK;
}

/* Index of the first angle of (set, round, pass) in the flat layout
   [set][round][pass][pair] (R N log2(N) / 2 angles per set, Sec. IV). */
static int64_t angle_offset(int log2n, int rounds, int set, int r, int p) {
  int64_t half = (int64_t)1 << (log2n - 1);
  return (((int64_t)set * rounds + r) * log2n + p) * half;
}

static int64_t perm_offset(int log2n, int rounds, int set, int r) {
  return ((int64_t)set * rounds + r) * ((int64_t)1 << log2n);
}

/* ------------------------------------------------------------------ */
/* Integer HyGT, one block.                                            */
/* ------------------------------------------------------------------ */
static int fwd_int_block(int log2n, int rounds, int set, const uint8_t *angle_idx,
                         const uint16_t *perms, const int32_t *ctab, const int32_t *stab,
                         int frac_bits, int64_t *v) {
  int N = 1 << log2n;
  int64_t half = (int64_t)1 << (frac_bits - 1);
  int64_t tmp[OR_MAX_N];
  for (int r = 0; r < rounds; ++r) {
    for (int p = 0; p < log2n; ++p) { /* one parallel-Givens pass */
      const uint8_t *q = angle_idx + angle_offset(log2n, rounds, set, r, p);
      for (int j = 0; j < N / 2; ++j) {
        int m, n;
        oracle_pair(p, j, &m, &n);
        int64_t c = ctab[q[j]], s = stab[q[j]];
        int64_t a = v[m], b = v[n];
        int64_t um = c * a + s * b + half;  /* row m of G(m,n,theta) */
        int64_t un = -s * a + c * b + half; /* row n of G(m,n,theta) */
        if (!fits_i32(um) || !fits_i32(un)) return OR_ERR_OVERFLOW;
        v[m] = floor_div_pow2(um, frac_bits);
        v[n] = floor_div_pow2(un, frac_bits);
      }
    }
    if (perms) { /* permutation slot after round r: gather */
      const uint16_t *pi = perms + perm_offset(log2n, rounds, set, r);
      for (int i = 0; i < N; ++i) tmp[i] = v[pi[i]];
      for (int i = 0; i < N; ++i) v[i] = tmp[i];
    }
  }
  return OR_OK;
}

static int inv_int_block(int log2n, int rounds, int set, const uint8_t *angle_idx,
                         const uint16_t *perms, const int32_t *ctab, const int32_t *stab,
                         int frac_bits, int64_t *v) {
  int N = 1 << log2n;
  int64_t half = (int64_t)1 << (frac_bits - 1);
  int64_t tmp[OR_MAX_N];
  for (int r = rounds - 1; r >= 0; --r) {
    if (perms) { /* undo the gather of slot r: scatter */
      const uint16_t *pi = perms + perm_offset(log2n, rounds, set, r);
      for (int i = 0; i < N; ++i) tmp[pi[i]] = v[i];
      for (int i = 0; i < N; ++i) v[i] = tmp[i];
    }
    for (int p = log2n - 1; p >= 0; --p) { /* passes in reverse order */
      const uint8_t *q = angle_idx + angle_offset(log2n, rounds, set, r, p);
      for (int j = 0; j < N / 2; ++j) {
        int m, n;
        oracle_pair(p, j, &m, &n);
        /* G(m,n,-theta): cos(-t) = c, sin(-t) = -s */
        int64_t c = ctab[q[j]], s = -(int64_t)stab[q[j]];
        int64_t a = v[m], b = v[n];
        int64_t um = c * a + s * b + half;
        int64_t un = -s * a + c * b + half;
        if (!fits_i32(um) || !fits_i32(un)) return OR_ERR_OVERFLOW;
        v[m] = floor_div_pow2(um, frac_bits);
        v[n] = floor_div_pow2(un, frac_bits);
      }
    }
  }
  return OR_OK;
}

/* Shared entry of the integer paths: validates the set index, calls the
   per-block routine, records the first error (lowest block index wins). */
int oracle_fwd_int(int log2n, int rounds, int num_sets, const uint8_t *angle_idx,
                   const uint16_t *perms, int angle_bits, int frac_bits,
                   const int16_t *x, const uint16_t *set_idx, int64_t nblocks, int32_t *y) {
  int st = check_shape(log2n, rounds, num_sets);
  if (st) return st;
  int32_t ctab[256], stab[256];
  st = oracle_cs_table(angle_bits, frac_bits, ctab, stab);
  if (st) return st;
  int N = 1 << log2n;
  int64_t first_bad = -1;
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t v[OR_MAX_N];
    unsigned set = set_idx ? set_idx[b] : 0u;
    int code = OR_OK;
    for (int i = 0; i < N; ++i) v[i] = x[b * N + i];
    if (set == OR_SKIP) {
      /* identity: widen */
    } else if (set >= (unsigned)num_sets) {
      code = OR_ERR_SET;
    } else {
      code = fwd_int_block(log2n, rounds, (int)set, angle_idx, perms, ctab, stab, frac_bits, v);
    }
    if (code != OR_OK) {
      for (int i = 0; i < N; ++i) v[i] = 0;
#pragma omp critical
      {
        if (first_bad < 0 || b < first_bad) { first_bad = b; bad_code = code; }
      }
    }
    for (int i = 0; i < N; ++i) y[b * N + i] = (int32_t)v[i];
  }
  return bad_code;
}

int oracle_inv_int(int log2n, int rounds, int num_sets, const uint8_t *angle_idx,
                   const uint16_t *perms, int angle_bits, int frac_bits,
                   const int32_t *y, const uint16_t *set_idx, int64_t nblocks, int16_t *x) {
  int st = check_shape(log2n, rounds, num_sets);
  if (st) return st;
  int32_t ctab[256], stab[256];
  st = oracle_cs_table(angle_bits, frac_bits, ctab, stab);
  if (st) return st;
  int N = 1 << log2n;
  int64_t first_bad = -1;
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t v[OR_MAX_N];
    unsigned set = set_idx ? set_idx[b] : 0u;
    int code = OR_OK;
    for (int i = 0; i < N; ++i) v[i] = y[b * N + i];
    if (set == OR_SKIP) {
      /* identity: narrow with saturation below */
    } else if (set >= (unsigned)num_sets) {
      code = OR_ERR_SET;
    } else {
      code = inv_int_block(log2n, rounds, (int)set, angle_idx, perms, ctab, stab, frac_bits, v);
    }
    if (code != OR_OK) {
      for (int i = 0; i < N; ++i) v[i] = 0;
#pragma omp critical
      {
        if (first_bad < 0 || b < first_bad) { first_bad = b; bad_code = code; }
      }
    }
    for (int i = 0; i < N; ++i) x[b * N + i] = saturate_i16(v[i]);
  }
  return bad_code;
}

/* ------------------------------------------------------------------ */
/* FP64 HyGT with free angles theta[set][round][pass][pair].           */
/* ------------------------------------------------------------------ */
static void fwd_f64_block(int log2n, int rounds, int set, const double *theta,
                          const uint16_t *perms, double *v) {
  int N = 1 << log2n;
  double tmp[OR_MAX_N];
  for (int r = 0; r < rounds; ++r) {
    for (int p = 0; p < log2n; ++p) {
      const double *t = theta + angle_offset(log2n, rounds, set, r, p);
      for (int j = 0; j < N / 2; ++j) {
        int m, n;
        oracle_pair(p, j, &m, &n);
        double c = cos(t[j]), s = sin(t[j]);
        double a = v[m], b = v[n];
        v[m] = c * a + s * b;
        v[n] = -s * a + c * b;
      }
    }
    if (perms) {
      const uint16_t *pi = perms + perm_offset(log2n, rounds, set, r);
      for (int i = 0; i < N; ++i) tmp[i] = v[pi[i]];
      for (int i = 0; i < N; ++i) v[i] = tmp[i];
    }
  }
}

static void inv_f64_block(int log2n, int rounds, int set, const double *theta,
                          const uint16_t *perms, double *v) {
  int N = 1 << log2n;
  double tmp[OR_MAX_N];
  for (int r = rounds - 1; r >= 0; --r) {
    if (perms) {
      const uint16_t *pi = perms + perm_offset(log2n, rounds, set, r);
      for (int i = 0; i < N; ++i) tmp[pi[i]] = v[i];
      for (int i = 0; i < N; ++i) v[i] = tmp[i];
    }
    for (int p = log2n - 1; p >= 0; --p) {
      const double *t = theta + angle_offset(log2n, rounds, set, r, p);
      for (int j = 0; j < N / 2; ++j) {
        int m, n;
        oracle_pair(p, j, &m, &n);
        double c = cos(-t[j]), s = sin(-t[j]);
        double a = v[m], b = v[n];
        v[m] = c * a + s * b;
        v[n] = -s * a + c * b;
      }
    }
  }
}

static int f64_run(int inverse, int log2n, int rounds, int num_sets, const double *theta,
                      const uint16_t *perms, const double *x, const uint16_t *set_idx,
                      int64_t nblocks, double *y) {
  int st = check_shape(log2n, rounds, num_sets);
  if (st) return st;
  int N = 1 << log2n;
  int64_t first_bad = -1;
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    double v[OR_MAX_N];
    unsigned set = set_idx ? set_idx[b] : 0u;
    for (int i = 0; i < N; ++i) v[i] = x[b * N + i];
    if (set == OR_SKIP) {
      /* identity */
    } else if (set >= (unsigned)num_sets) {
      for (int i = 0; i < N; ++i) v[i] = 0.0;
#pragma omp critical
      {
        if (first_bad < 0 || b < first_bad) { first_bad = b; bad_code = OR_ERR_SET; }
      }
    } else if (inverse) {
      inv_f64_block(log2n, rounds, (int)set, theta, perms, v);
    } else {
      fwd_f64_block(log2n, rounds, (int)set, theta, perms, v);
    }
    for (int i = 0; i < N; ++i) y[b * N + i] = v[i];
  }
  return bad_code;
}

int oracle_fwd_f64(int log2n, int rounds, int num_sets, const double *theta, const uint16_t *perms,
                   const double *x, const uint16_t *set_idx, int64_t nblocks, double *y) {
  return f64_run(0, log2n, rounds, num_sets, theta, perms, x, set_idx, nblocks, y);
}

int oracle_inv_f64(int log2n, int rounds, int num_sets, const double *theta, const uint16_t *perms,
                   const double *y, const uint16_t *set_idx, int64_t nblocks, double *x) {
  return f64_run(1, log2n, rounds, num_sets, theta, perms, y, set_idx, nblocks, x);
}

/* Dense N x N matrix T of one set (row-major, T[i*N + k]): column k is the
   transform of the unit vector e_k (PMPT product, Eq. 5). */
int oracle_dense_f64(int log2n, int rounds, const double *theta_set, const uint16_t *perms_set,
                     double *T) {
  int st = check_shape(log2n, rounds, 1);
  if (st) return st;
  int N = 1 << log2n;
  double v[OR_MAX_N];
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i < N; ++i) v[i] = (i == k) ? 1.0 : 0.0;
    fwd_f64_block(log2n, rounds, 0, theta_set, perms_set, v);
    for (int i = 0; i < N; ++i) T[i * N + k] = v[i];
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Energy-compaction loss and its analytic gradient (one set).         */
/* L = (1/B) sum_b sum_{i >= K} y_{b,i}^2,  y_b = T(theta) x_b.        */
/* The gradient back-propagates through the stored FP64 input of every */
/* pass: for a rotation (a,b) -> (c a + s b, -s a + c b),               */
/*   dL/dtheta += g_m * (-s a + c b) + g_n * (-c a - s b),              */
/*   dL/da = c g_m - s g_n,   dL/db = s g_m + c g_n,                    */
/* and through a gather slot v'[i] = v[pi[i]] by g_v[pi[i]] += g_v'[i]. */
/* gtheta has the layout of theta; gx (nullable) has the layout of x.   */
/* ------------------------------------------------------------------ */
int oracle_loss_grad_f64(int log2n, int rounds, const double *theta, const uint16_t *perms,
                         const double *x, int64_t nblocks, int K, double *loss,
                         double *gtheta, double *gx) {
  int st = check_shape(log2n, rounds, 1);
  if (st) return st;
  int N = 1 << log2n;
  if (K < 0 || K > N || nblocks < 1) return OR_ERR_ARG;
  int P = rounds * log2n;
  int64_t nangles = (int64_t)P * (N / 2);
  int nth = oracle_num_threads();
  double *gacc = (double *)calloc((size_t)nth * (size_t)nangles, sizeof(double));
  double *lacc = (double *)calloc((size_t)nth, sizeof(double));
  if (!gacc || !lacc) { free(gacc); free(lacc); return OR_ERR_ARG; }
  double inv_b = 1.0 / (double)nblocks;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double *gt = gacc + (size_t)tid * (size_t)nangles;
    /* stored activations: the input of every pass and of every perm slot */
    double *act = (double *)malloc(sizeof(double) * (size_t)(P + rounds + 1) * (size_t)N);
#pragma omp for schedule(static)
    for (int64_t b = 0; b < nblocks; ++b) {
      double v[OR_MAX_N], g[OR_MAX_N], tmp[OR_MAX_N];
      for (int i = 0; i < N; ++i) v[i] = x[b * N + i];
      int slot = 0;
      for (int r = 0; r < rounds; ++r) {
        for (int p = 0; p < log2n; ++p) {
          memcpy(act + (size_t)slot * N, v, sizeof(double) * N);
          ++slot;
          const double *t = theta + angle_offset(log2n, rounds, 0, r, p);
          for (int j = 0; j < N / 2; ++j) {
            int m, n;
            oracle_pair(p, j, &m, &n);
            double c = cos(t[j]), s = sin(t[j]);
            double a = v[m], bb = v[n];
            v[m] = c * a + s * bb;
            v[n] = -s * a + c * bb;
          }
        }
        if (perms) {
          const uint16_t *pi = perms + perm_offset(log2n, rounds, 0, r);
          for (int i = 0; i < N; ++i) tmp[i] = v[pi[i]];
          for (int i = 0; i < N; ++i) v[i] = tmp[i];
        }
      }
      double l = 0.0;
      for (int i = 0; i < N; ++i) {
        if (i >= K) {
          l += v[i] * v[i];
          g[i] = 2.0 * v[i] * inv_b;
        } else {
          g[i] = 0.0;
        }
      }
      lacc[tid] += l * inv_b;
      for (int r = rounds - 1; r >= 0; --r) {
        if (perms) {
          const uint16_t *pi = perms + perm_offset(log2n, rounds, 0, r);
          for (int i = 0; i < N; ++i) tmp[i] = 0.0;
          for (int i = 0; i < N; ++i) tmp[pi[i]] += g[i];
          for (int i = 0; i < N; ++i) g[i] = tmp[i];
        }
        for (int p = log2n - 1; p >= 0; --p) {
          --slot;
          const double *in = act + (size_t)slot * N;
          const double *t = theta + angle_offset(log2n, rounds, 0, r, p);
          double *gtp = gt + angle_offset(log2n, rounds, 0, r, p);
          for (int j = 0; j < N / 2; ++j) {
            int m, n;
            oracle_pair(p, j, &m, &n);
            double c = cos(t[j]), s = sin(t[j]);
            double a = in[m], bb = in[n];
            double gm = g[m], gn = g[n];
            gtp[j] += gm * (-s * a + c * bb) + gn * (-c * a - s * bb);
            g[m] = c * gm - s * gn;
            g[n] = s * gm + c * gn;
          }
        }
      }
      if (gx)
        for (int i = 0; i < N; ++i) gx[b * N + i] = g[i];
    }
    free(act);
  }
  double L = 0.0;
  for (int t = 0; t < nth; ++t) L += lacc[t];
  for (int64_t a = 0; a < nangles; ++a) {
    double sum = 0.0;
    for (int t = 0; t < nth; ++t) sum += gacc[(size_t)t * (size_t)nangles + (size_t)a];
    gtheta[a] = sum;
  }
  *loss = L;
  free(gacc);
  free(lacc);
  return OR_OK;
}

/* Loss only (for finite differences). */
int oracle_loss_f64(int log2n, int rounds, const double *theta, const uint16_t *perms,
                    const double *x, int64_t nblocks, int K, double *loss) {
  int st = check_shape(log2n, rounds, 1);
  if (st) return st;
  int N = 1 << log2n;
  if (K < 0 || K > N || nblocks < 1) return OR_ERR_ARG;
  double total = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : total)
  for (int64_t b = 0; b < nblocks; ++b) {
    double v[OR_MAX_N];
    for (int i = 0; i < N; ++i) v[i] = x[b * N + i];
    fwd_f64_block(log2n, rounds, 0, theta, perms, v);
    double l = 0.0;
    for (int i = K; i < N; ++i) l += v[i] * v[i];
    total += l;
  }
  *loss = total / (double)nblocks;
  return OR_OK;
}

/* Dense per-block matrix product (the matrix transform of Eq. 3),
   y_b = K_{set(b)} x_b in FP64, K as [num_sets][N][N] row-major. */
int oracle_dense_apply_f64(int n, int num_sets, const double *K, const double *x,
                           const uint16_t *set_idx, int64_t nblocks, double *y) {
  if (n < 1 || n > OR_MAX_N || num_sets < 1) return OR_ERR_ARG;
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    unsigned set = set_idx ? set_idx[b] : 0u;
    if (set == OR_SKIP) {
      for (int i = 0; i < n; ++i) y[b * n + i] = x[b * n + i];
      continue;
    }
    if (set >= (unsigned)num_sets) {
      for (int i = 0; i < n; ++i) y[b * n + i] = 0.0;
#pragma omp critical
      bad_code = OR_ERR_SET;
      continue;
    }
    const double *M = K + (size_t)set * n * n;
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += M[i * n + k] * x[b * n + k];
      y[b * n + i] = acc;
    }
  }
  return bad_code;
}

/* Integer matrix transform: y_b = floor((K_int x_b + 2^(f-1)) / 2^f),
   K_int as int32 [num_sets][N][N]; int64 accumulation, checked to fit int32. */
int oracle_dense_apply_int(int n, int num_sets, const int32_t *K, int frac_bits, const int16_t *x,
                           const uint16_t *set_idx, int64_t nblocks, int32_t *y) {
  if (n < 1 || n > OR_MAX_N || num_sets < 1 || frac_bits < 1 || frac_bits > 14) return OR_ERR_ARG;
  int64_t half = (int64_t)1 << (frac_bits - 1);
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    unsigned set = set_idx ? set_idx[b] : 0u;
    if (set == OR_SKIP) {
      for (int i = 0; i < n; ++i) y[b * n + i] = x[b * n + i];
      continue;
    }
    if (set >= (unsigned)num_sets) {
      for (int i = 0; i < n; ++i) y[b * n + i] = 0;
#pragma omp critical
      bad_code = OR_ERR_SET;
      continue;
    }
    const int32_t *M = K + (size_t)set * n * n;
    for (int i = 0; i < n; ++i) {
      int64_t acc = half;
      for (int k = 0; k < n; ++k) acc += (int64_t)M[i * n + k] * (int64_t)x[b * n + k];
      if (!fits_i32(acc)) {
#pragma omp critical
        bad_code = OR_ERR_OVERFLOW;
      }
      y[b * n + i] = (int32_t)floor_div_pow2(acc, frac_bits);
    }
  }
  return bad_code;
}

/* ------------------------------------------------------------------ */
/* General PMPT with explicit index vectors (Sec. III PMPT product,    */
/* Eq. 5; Sec. IV parallel-Givens matrix over an arbitrary pair cover, */
/* Eq. 7 and Eq. 8).  Pass k of set s has N/2 pairs (m_j, n_j) and N/2 */
/* angles; the pairs must cover 0..N-1 (each index in exactly one      */
/* pair), which makes the rotations of a pass commute.  Layouts:       */
/* angles [S][P][N/2] (8-bit indices or FP64 radians), m and n         */
/* [S][P][N/2].  N is any even number up to 256.  The forward applies  */
/* pass 0 first; the inverse runs the passes in reverse with negated   */
/* angles (Eq. 9).  Integer rounding, skip and bad-set handling are    */
/* those of the HyGT paths above.                                      */
/* ------------------------------------------------------------------ */
static int pmpt_check(int n, int passes, int num_sets, const uint16_t *m_idx,
                      const uint16_t *n_idx) {
  if (n < 2 || n > OR_MAX_N || (n & 1) || passes < 1 || passes > 4096) return OR_ERR_ARG;
  if (num_sets < 1 || num_sets > 65535 || !m_idx || !n_idx) return OR_ERR_ARG;
  for (int64_t sp = 0; sp < (int64_t)num_sets * passes; ++sp) {
    int seen[OR_MAX_N];
    memset(seen, 0, sizeof(seen));
    for (int j = 0; j < n / 2; ++j) {
      int m = m_idx[sp * (n / 2) + j], k = n_idx[sp * (n / 2) + j];
      if (m >= n || k >= n || m == k || seen[m] || seen[k]) return OR_ERR_ARG;
      seen[m] = seen[k] = 1;
    }
  }
  return OR_OK;
}

static int pmpt_int_block(int inverse, int n, int passes, int set, const uint8_t *angle_idx,
                          const uint16_t *m_idx, const uint16_t *n_idx, const int32_t *ctab,
                          const int32_t *stab, int frac_bits, int64_t *v) {
  int64_t half = (int64_t)1 << (frac_bits - 1);
  for (int kk = 0; kk < passes; ++kk) {
    int k = inverse ? passes - 1 - kk : kk;
    int64_t base = ((int64_t)set * passes + k) * (n / 2);
    for (int j = 0; j < n / 2; ++j) {
      int m = m_idx[base + j], q = n_idx[base + j];
      int64_t c = ctab[angle_idx[base + j]];
      int64_t s = inverse ? -(int64_t)stab[angle_idx[base + j]] : stab[angle_idx[base + j]];
      int64_t a = v[m], b = v[q];
      int64_t um = c * a + s * b + half;
      int64_t un = -s * a + c * b + half;
      if (!fits_i32(um) || !fits_i32(un)) return OR_ERR_OVERFLOW;
      v[m] = floor_div_pow2(um, frac_bits);
      v[q] = floor_div_pow2(un, frac_bits);
    }
  }
  return OR_OK;
}

static int pmpt_int_run(int inverse, int n, int passes, int num_sets, const uint8_t *angle_idx,
                        const uint16_t *m_idx, const uint16_t *n_idx, int angle_bits,
                        int frac_bits, const void *in, const uint16_t *set_idx, int64_t nblocks,
                        void *out) {
  int st = pmpt_check(n, passes, num_sets, m_idx, n_idx);
  if (st) return st;
  int32_t ctab[256], stab[256];
  st = oracle_cs_table(angle_bits, frac_bits, ctab, stab);
  if (st) return st;
  int64_t first_bad = -1;
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t v[OR_MAX_N];
    unsigned set = set_idx ? set_idx[b] : 0u;
    int code = OR_OK;
    for (int i = 0; i < n; ++i)
      v[i] = inverse ? ((const int32_t *)in)[b * n + i] : ((const int16_t *)in)[b * n + i];
    if (set == OR_SKIP) {
      /* identity */
    } else if (set >= (unsigned)num_sets) {
      code = OR_ERR_SET;
    } else {
      code = pmpt_int_block(inverse, n, passes, (int)set, angle_idx, m_idx, n_idx, ctab, stab,
                            frac_bits, v);
    }
    if (code != OR_OK) {
      for (int i = 0; i < n; ++i) v[i] = 0;
#pragma omp critical
      {
        if (first_bad < 0 || b < first_bad) { first_bad = b; bad_code = code; }
      }
    }
    for (int i = 0; i < n; ++i) {
      if (inverse) ((int16_t *)out)[b * n + i] = saturate_i16(v[i]);
      else ((int32_t *)out)[b * n + i] = (int32_t)v[i];
    }
  }
  return bad_code;
}

int oracle_pmpt_fwd_int(int n, int passes, int num_sets, const uint8_t *angle_idx,
                        const uint16_t *m_idx, const uint16_t *n_idx, int angle_bits,
                        int frac_bits, const int16_t *x, const uint16_t *set_idx,
                        int64_t nblocks, int32_t *y) {
  return pmpt_int_run(0, n, passes, num_sets, angle_idx, m_idx, n_idx, angle_bits, frac_bits, x,
                      set_idx, nblocks, y);
}

int oracle_pmpt_inv_int(int n, int passes, int num_sets, const uint8_t *angle_idx,
                        const uint16_t *m_idx, const uint16_t *n_idx, int angle_bits,
                        int frac_bits, const int32_t *y, const uint16_t *set_idx,
                        int64_t nblocks, int16_t *x) {
  return pmpt_int_run(1, n, passes, num_sets, angle_idx, m_idx, n_idx, angle_bits, frac_bits, y,
                      set_idx, nblocks, x);
}

static int pmpt_f64_run(int inverse, int n, int passes, int num_sets, const double *theta,
                        const uint16_t *m_idx, const uint16_t *n_idx, const double *in,
                        const uint16_t *set_idx, int64_t nblocks, double *out) {
  int st = pmpt_check(n, passes, num_sets, m_idx, n_idx);
  if (st) return st;
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    double v[OR_MAX_N];
    unsigned set = set_idx ? set_idx[b] : 0u;
    for (int i = 0; i < n; ++i) v[i] = in[b * n + i];
    if (set != OR_SKIP && set >= (unsigned)num_sets) {
      for (int i = 0; i < n; ++i) v[i] = 0.0;
#pragma omp critical
      bad_code = OR_ERR_SET;
    } else if (set != OR_SKIP) {
      for (int kk = 0; kk < passes; ++kk) {
        int k = inverse ? passes - 1 - kk : kk;
        int64_t base = ((int64_t)set * passes + k) * (n / 2);
        for (int j = 0; j < n / 2; ++j) {
          int m = m_idx[base + j], q = n_idx[base + j];
          double t = inverse ? -theta[base + j] : theta[base + j];
          double c = cos(t), s = sin(t);
          double a = v[m], bb = v[q];
          v[m] = c * a + s * bb;
          v[q] = -s * a + c * bb;
        }
      }
    }
    for (int i = 0; i < n; ++i) out[b * n + i] = v[i];
  }
  return bad_code;
}

int oracle_pmpt_fwd_f64(int n, int passes, int num_sets, const double *theta,
                        const uint16_t *m_idx, const uint16_t *n_idx, const double *x,
                        const uint16_t *set_idx, int64_t nblocks, double *y) {
  return pmpt_f64_run(0, n, passes, num_sets, theta, m_idx, n_idx, x, set_idx, nblocks, y);
}

int oracle_pmpt_inv_f64(int n, int passes, int num_sets, const double *theta,
                        const uint16_t *m_idx, const uint16_t *n_idx, const double *y,
                        const uint16_t *set_idx, int64_t nblocks, double *x) {
  return pmpt_f64_run(1, n, passes, num_sets, theta, m_idx, n_idx, y, set_idx, nblocks, x);
}

/* ------------------------------------------------------------------ */
/* Secondary-transform pipeline (Sec. VI): a separable primary         */
/* transform of an M x M residual block, then the HyGT on the top-left */
/* s x s sub-block of its coefficients (s = 4 for 4 x 4 blocks, s = 8  */
/* for 8 x 8 and larger), the other coefficients passed through.  The  */
/* paper does not fix the primary; it is read here as the orthonormal  */
/* 2-D DCT-II, D[k][i] = a_k cos(pi (2i + 1) k / (2M)) with            */
/* a_0 = sqrt(1/M), a_k = sqrt(2/M), in integer arithmetic with the    */
/* HyGT's precision: C = round(2^8 D) (half away from zero), each 1-D  */
/* stage y_k = floor((sum_i C[k][i] x_i + 2^7) / 2^8), rows first then */
/* columns; the inverse runs the columns first, then the rows, with    */
/* C transposed and the same rounding, and saturates to int16.  The    */
/* sub-block is read in raster order (the HyGT's vector order).  Set   */
/* index 0xFFFF means "no secondary transform" (primary only).         */
/* ------------------------------------------------------------------ */
#define OR_PRIMARY_BITS 8
#define OR_MAX_M 32

/* FP64 DCT-II matrix and its integer form [M][M] (row k = basis k). */
int oracle_dct_matrix(int log2m, int32_t *C, double *D) {
  if (log2m < 1 || log2m > 5) return OR_ERR_ARG;
  int M = 1 << log2m;
  double scale = ldexp(1.0, OR_PRIMARY_BITS);
  for (int k = 0; k < M; ++k) {
    double a = k == 0 ? sqrt(1.0 / M) : sqrt(2.0 / M);
    for (int i = 0; i < M; ++i) {
      double d = a * cos(OR_TWO_PI * 0.5 * (2.0 * i + 1.0) * k / (2.0 * M));
      if (D) D[k * M + i] = d;
      if (C) C[k * M + i] = (int32_t)lround(scale * d);
    }
  }
  return OR_OK;
}

/* One separable stage along rows (dim 0) or columns (dim 1) of an M x M
   block held row-major in v; transpose selects C^T (inverse).  Returns
   OR_ERR_OVERFLOW when a sum leaves int32 (the range the integer
   arithmetic is specified for, as for the HyGT butterflies). */
static int primary_stage(int M, const int32_t *C, int dim, int transpose, int64_t *v) {
  int64_t half = (int64_t)1 << (OR_PRIMARY_BITS - 1);
  int64_t line[OR_MAX_M], out[OR_MAX_M];
  for (int l = 0; l < M; ++l) {
    for (int i = 0; i < M; ++i) line[i] = dim == 0 ? v[l * M + i] : v[i * M + l];
    for (int k = 0; k < M; ++k) {
      int64_t acc = half;
      for (int i = 0; i < M; ++i)
        acc += (int64_t)(transpose ? C[i * M + k] : C[k * M + i]) * line[i];
      if (!fits_i32(acc)) return OR_ERR_OVERFLOW;
      out[k] = floor_div_pow2(acc, OR_PRIMARY_BITS);
    }
    for (int k = 0; k < M; ++k) {
      if (dim == 0) v[l * M + k] = out[k];
      else v[k * M + l] = out[k];
    }
  }
  return OR_OK;
}

static int secondary_run(int inverse, int log2m, int log2n, int rounds, int num_sets,
                         const uint8_t *angle_idx, const uint16_t *perms, int angle_bits,
                         int frac_bits, const void *in, const uint16_t *set_idx, int64_t nblocks,
                         void *out) {
  int st = check_shape(log2n, rounds, num_sets);
  if (st) return st;
  if (log2m < 2 || log2m > 5 || (log2n != 4 && log2n != 6)) return OR_ERR_ARG;
  int M = 1 << log2m, s = 1 << (log2n / 2);
  if ((M == 4 && s != 4) || (M >= 8 && s != 8)) return OR_ERR_ARG;
  int32_t C[OR_MAX_M * OR_MAX_M];
  oracle_dct_matrix(log2m, C, NULL);
  int32_t ctab[256], stab[256];
  st = oracle_cs_table(angle_bits, frac_bits, ctab, stab);
  if (st) return st;
  int64_t first_bad = -1;
  int bad_code = OR_OK;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t v[OR_MAX_M * OR_MAX_M], sub[OR_MAX_N];
    unsigned set = set_idx ? set_idx[b] : 0u;
    int code = OR_OK;
    int MM = M * M;
    for (int i = 0; i < MM; ++i)
      v[i] = inverse ? ((const int32_t *)in)[b * MM + i] : ((const int16_t *)in)[b * MM + i];
    if (set != OR_SKIP && set >= (unsigned)num_sets) code = OR_ERR_SET;
    if (code == OR_OK && !inverse) {
      code = primary_stage(M, C, 0, 0, v);             /* rows */
      if (code == OR_OK) code = primary_stage(M, C, 1, 0, v); /* columns */
    }
    if (code == OR_OK && set != OR_SKIP) {
      for (int r = 0; r < s; ++r)
        for (int c = 0; c < s; ++c) sub[r * s + c] = v[r * M + c];
      code = inverse ? inv_int_block(log2n, rounds, (int)set, angle_idx, perms, ctab, stab,
                                     frac_bits, sub)
                     : fwd_int_block(log2n, rounds, (int)set, angle_idx, perms, ctab, stab,
                                     frac_bits, sub);
      for (int r = 0; r < s; ++r)
        for (int c = 0; c < s; ++c) v[r * M + c] = sub[r * s + c];
    }
    if (code == OR_OK && inverse) {
      code = primary_stage(M, C, 1, 1, v);             /* columns */
      if (code == OR_OK) code = primary_stage(M, C, 0, 1, v); /* rows */
    }
    if (code == OR_OK) {
      for (int i = 0; i < MM; ++i)
        if (!fits_i32(v[i])) code = OR_ERR_OVERFLOW;
    }
    if (code != OR_OK) {
      for (int i = 0; i < MM; ++i) v[i] = 0;
#pragma omp critical
      {
        if (first_bad < 0 || b < first_bad) { first_bad = b; bad_code = code; }
      }
    }
    for (int i = 0; i < MM; ++i) {
      if (inverse) ((int16_t *)out)[b * MM + i] = saturate_i16(v[i]);
      else ((int32_t *)out)[b * MM + i] = (int32_t)v[i];
    }
  }
  return bad_code;
}

int oracle_secondary_fwd(int log2m, int log2n, int rounds, int num_sets,
                         const uint8_t *angle_idx, const uint16_t *perms, int angle_bits,
                         int frac_bits, const int16_t *x, const uint16_t *set_idx,
                         int64_t nblocks, int32_t *y) {
  return secondary_run(0, log2m, log2n, rounds, num_sets, angle_idx, perms, angle_bits,
                       frac_bits, x, set_idx, nblocks, y);
}

int oracle_secondary_inv(int log2m, int log2n, int rounds, int num_sets,
                         const uint8_t *angle_idx, const uint16_t *perms, int angle_bits,
                         int frac_bits, const int32_t *y, const uint16_t *set_idx,
                         int64_t nblocks, int16_t *x) {
  return secondary_run(1, log2m, log2n, rounds, num_sets, angle_idx, perms, angle_bits,
                       frac_bits, y, set_idx, nblocks, x);
}
