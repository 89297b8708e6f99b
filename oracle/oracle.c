/*
 * oracle.c -- plain, slow, obviously correct CPU definition of the X-engine.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares
 * no code, header or table with the CUDA path.
 *
 * Definitions followed (paper: "Design and Implementation of a Scalable
 * Correlator Based on ROACH2+GPU Cluster for Tianlai 96-Dual-Polarization
 * Antenna Array"):
 *   - Sec. 2.1 (F-engine): each complex sample is a 4-bit real part and a
 *     4-bit imaginary part.  Reading adopted here: one byte per sample, high
 *     nibble = real, low nibble = imaginary, each 4-bit two's complement
 *     (range -8..7).
 *   - Sec. 2.3 (X-engine): the X-engine performs conjugate multiplication and
 *     accumulation (CMAC) per frequency channel over all input pairs
 *     (baselines).
 *   - Eq. 1 (Sec. 2.2): N inputs give N(N+1)/2 products per channel, i.e. the
 *     lower triangle of the correlation matrix including the autos.
 *   - Eq. 2 (Sec. 3.2): a visibility is the time average of the product of one
 *     signal with the conjugate of the other.  Reading adopted here: the
 *     stored element for i >= j is V[i][j] = sum_t x_i(t) * conj(x_j(t)),
 *     which is Eq. 2's <S1^* S2> with S1 = x_j and S2 = x_i.  No averaging:
 *     the integer sum is kept (int64).
 *   - Sec. 1 / abstract: "full-Stokes output".  The paper gives no formula.
 *     Reading adopted here, per antenna pair (p >= q), with input index
 *     i = 2*antenna + pol (pol 0 = X, 1 = Y):
 *         XX = V[2p][2q], YY = V[2p+1][2q+1], XY = V[2p][2q+1], YX = V[2p+1][2q]
 *         (for p == q the XY element lies above the diagonal and is taken as
 *          conj(V[2p+1][2p]))
 *         I = XX + YY, Q = XX - YY, U = XY + YX, V = -j (XY - YX)
 *     all integer, no factor 1/2.
 *
 * Layouts:
 *   x      uint8  [n_chan][n_in][T]
 *   vis    int64  [n_chan][P][2]     P = n_in(n_in+1)/2, pair index i(i+1)/2 + j
 *   full   int64  [n_chan][n_in][n_in][2]  (every i, j; Hermitian check)
 *   stokes int64  [n_chan][A][4][2]  A = n_ant(n_ant+1)/2, pair index p(p+1)/2 + q,
 *                                    order I, Q, U, V; (re, im)
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

/* 4-bit two's complement nibble -> integer in [-8, 7] */
static int64_t nibble_value(unsigned v) {
  v &= 15u;
  return v >= 8u ? (int64_t)v - 16 : (int64_t)v;
}

void oracle_decode(uint8_t b, int64_t *re, int64_t *im) {
  *re = nibble_value((unsigned)b >> 4);
  *im = nibble_value((unsigned)b);
}

/* V[i][j] for one channel, any i, j: sum_t x_i(t) conj(x_j(t)). */
static void cmac_pair(const uint8_t *xi, const uint8_t *xj, int T, int64_t *re_out,
                      int64_t *im_out) {
  int64_t re = 0, im = 0;
  for (int t = 0; t < T; ++t) {
    int64_t ai, bi, aj, bj;
    oracle_decode(xi[t], &ai, &bi);
    oracle_decode(xj[t], &aj, &bj);
    /* (ai + j bi)(aj - j bj) = (ai aj + bi bj) + j (bi aj - ai bj) */
    re += ai * aj + bi * bj;
    im += bi * aj - ai * bj;
  }
  *re_out = re;
  *im_out = im;
}

typedef struct {
  const uint8_t *x;
  int n_in, T, c_lo, c_hi;
  int64_t *vis;
} xjob_t;

static void *xcorr_range(void *arg) {
  const xjob_t *jb = (const xjob_t *)arg;
  const size_t P = (size_t)jb->n_in * (size_t)(jb->n_in + 1) / 2;
  for (int c = jb->c_lo; c < jb->c_hi; ++c) {
    const uint8_t *xc = jb->x + (size_t)c * jb->n_in * (size_t)jb->T;
    int64_t *vc = jb->vis + (size_t)c * P * 2;
    for (int i = 0; i < jb->n_in; ++i) {
      for (int j = 0; j <= i; ++j) {
        int64_t re, im;
        cmac_pair(xc + (size_t)i * jb->T, xc + (size_t)j * jb->T, jb->T, &re, &im);
        size_t p = (size_t)i * (size_t)(i + 1) / 2 + (size_t)j;
        vc[2 * p] += re;
        vc[2 * p + 1] += im;
      }
    }
  }
  return NULL;
}

/*
 * Accumulates (+=) the lower-triangle visibilities of one block into vis.
 * Channels are split over n_threads plain threads (each channel is written
 * by exactly one thread).  Returns 0, or -1 on bad arguments.
 */
int oracle_xcorr(const uint8_t *x, int n_in, int n_chan, int T, int64_t *vis, int n_threads) {
  if (!x || !vis || n_in <= 0 || n_chan <= 0 || T < 0) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_chan) n_threads = n_chan;
  xjob_t *jobs = (xjob_t *)calloc((size_t)n_threads, sizeof(xjob_t));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -1; }
  for (int k = 0; k < n_threads; ++k) {
    jobs[k].x = x; jobs[k].n_in = n_in; jobs[k].T = T; jobs[k].vis = vis;
    jobs[k].c_lo = (int)((long long)n_chan * k / n_threads);
    jobs[k].c_hi = (int)((long long)n_chan * (k + 1) / n_threads);
  }
  int started = 0;
  for (int k = 1; k < n_threads; ++k) {
    if (pthread_create(&th[k], NULL, xcorr_range, &jobs[k]) != 0) break;
    started = k;
  }
  xcorr_range(&jobs[0]);
  for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
  for (int k = started + 1; k < n_threads; ++k) xcorr_range(&jobs[k]);
  free(jobs); free(th);
  return 0;
}

/* One pair (i, j) of one channel: the sampled check used at full sizes. */
int oracle_xcorr_pair(const uint8_t *x, int n_in, int T, int c, int i, int j, int64_t out[2]) {
  if (!x || !out || i < 0 || j < 0 || i >= n_in || j >= n_in || c < 0 || T < 0) return -1;
  const uint8_t *xc = x + (size_t)c * n_in * (size_t)T;
  cmac_pair(xc + (size_t)i * T, xc + (size_t)j * T, T, &out[0], &out[1]);
  return 0;
}

/* Every (i, j), including the upper triangle, for the Hermitian check. */
int oracle_xcorr_full(const uint8_t *x, int n_in, int n_chan, int T, int64_t *full) {
  if (!x || !full || n_in <= 0 || n_chan <= 0 || T < 0) return -1;
  for (int c = 0; c < n_chan; ++c) {
    const uint8_t *xc = x + (size_t)c * n_in * (size_t)T;
    for (int i = 0; i < n_in; ++i)
      for (int j = 0; j < n_in; ++j) {
        int64_t *o = full + (((size_t)c * n_in + i) * n_in + j) * 2;
        cmac_pair(xc + (size_t)i * T, xc + (size_t)j * T, T, &o[0], &o[1]);
      }
  }
  return 0;
}

/* Element (i, j) of one channel's Hermitian matrix from the stored lower triangle. */
static void herm_get(const int64_t *vc, int i, int j, int64_t *re, int64_t *im) {
  if (i >= j) {
    size_t p = (size_t)i * (size_t)(i + 1) / 2 + (size_t)j;
    *re = vc[2 * p];
    *im = vc[2 * p + 1];
  } else {
    size_t p = (size_t)j * (size_t)(j + 1) / 2 + (size_t)i;
    *re = vc[2 * p];
    *im = -vc[2 * p + 1];
  }
}

/*
 * Full-Stokes products per antenna pair from dual-polarisation visibilities
 * (n_in = 2 * n_ant).  Writes (=) stokes[c][a][s][2], s = I, Q, U, V.
 */
int oracle_stokes(const int64_t *vis, int n_ant, int n_chan, int64_t *stokes) {
  if (!vis || !stokes || n_ant <= 0 || n_chan <= 0) return -1;
  const int n_in = 2 * n_ant;
  const size_t P = (size_t)n_in * (size_t)(n_in + 1) / 2;
  const size_t A = (size_t)n_ant * (size_t)(n_ant + 1) / 2;
  for (int c = 0; c < n_chan; ++c) {
    const int64_t *vc = vis + (size_t)c * P * 2;
    for (int p = 0; p < n_ant; ++p) {
      for (int q = 0; q <= p; ++q) {
        int64_t xx_r, xx_i, yy_r, yy_i, xy_r, xy_i, yx_r, yx_i;
        herm_get(vc, 2 * p, 2 * q, &xx_r, &xx_i);
        herm_get(vc, 2 * p + 1, 2 * q + 1, &yy_r, &yy_i);
        herm_get(vc, 2 * p, 2 * q + 1, &xy_r, &xy_i);
        herm_get(vc, 2 * p + 1, 2 * q, &yx_r, &yx_i);
        int64_t *s = stokes + ((size_t)c * A + (size_t)p * (size_t)(p + 1) / 2 + (size_t)q) * 8;
        s[0] = xx_r + yy_r;  s[1] = xx_i + yy_i;   /* I = XX + YY */
        s[2] = xx_r - yy_r;  s[3] = xx_i - yy_i;   /* Q = XX - YY */
        s[4] = xy_r + yx_r;  s[5] = xy_i + yx_i;   /* U = XY + YX */
        /* V = -j (XY - YX): -j (d_r + j d_i) = d_i - j d_r */
        s[6] = xy_i - yx_i;  s[7] = -(xy_r - yx_r);
      }
    }
  }
  return 0;
}
