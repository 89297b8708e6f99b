/*
 * synth.c -- seeded synthetic channelised voltages for the X-engine.
 *
 * This module only draws inputs.  It holds none of the correlator's
 * arithmetic: both the CUDA path and the CPU oracle consume the bytes it
 * writes, and neither imports the other.
 *
 * Sample model (the F-engine output format of Sec. 2.1: every complex
 * sample is a 4-bit real part and a 4-bit imaginary part after EQ and
 * requantisation):
 *
 *   z(c, i, t) = n(c, i, t) + sum_k amp_k * exp(j * (2*pi*f_k*t_abs
 *                                               + phase_k[i] + slope_k[i]*c))
 *   re = clip(round_half_away(Re z), -7, 7),  im = likewise for Im z
 *   byte = ((re & 15) << 4) | (im & 15)        (high nibble = real part)
 *
 * n is complex Gaussian noise with standard deviation sigma per component,
 * drawn by the Box-Muller transform from two uniforms produced by the
 * counter-based generator Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11).  The counter is
 * (t_abs low word, t_abs high word, input, channel) and the key is the
 * 64-bit seed, so every sample is a pure function of its coordinates and
 * the output does not depend on the thread count.  t_abs = block*T + t is
 * the sample index since the start of the stream, so consecutive blocks
 * continue each tone coherently.  slope_k[i]*c is a phase that grows
 * linearly with the channel index, as a cable delay does (Eq. 2).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

/* Philox4x32 with 10 rounds; ctr is updated in place to the output. */
void synth_philox4x32_10(uint32_t ctr[4], const uint32_t key_in[2]) {
  uint32_t k0 = key_in[0], k1 = key_in[1];
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += PHILOX_W0; k1 += PHILOX_W1;
  }
  ctr[0] = c0; ctr[1] = c1; ctr[2] = c2; ctr[3] = c3;
}

static int clip7(double v) {
  /* round half away from zero, then clip to the configured range */
  double r = v < 0.0 ? -floor(-v + 0.5) : floor(v + 0.5);
  if (r > 7.0) r = 7.0;
  if (r < -7.0) r = -7.0;
  return (int)r;
}

typedef struct {
  uint8_t *out;
  int n_in, n_chan, T, c0, chan_lo, chan_hi;
  uint64_t seed, block;
  double sigma;
  int n_tones;
  const double *amp, *freq, *phase, *slope; /* [n_tones], [n_tones], [n_tones*n_in] x2 */
} job_t;

static void *work(void *arg) {
  const job_t *j = (const job_t *)arg;
  const double two_pi = 6.283185307179586476925286766559;
  const double inv53 = 1.0 / 9007199254740992.0; /* 2^-53 */
  uint32_t key[2] = {(uint32_t)j->seed, (uint32_t)(j->seed >> 32)};
  for (int cl = j->chan_lo; cl < j->chan_hi; ++cl) {
    int c = j->c0 + cl; /* global channel index */
    for (int i = 0; i < j->n_in; ++i) {
      uint8_t *row = j->out + ((size_t)cl * j->n_in + i) * (size_t)j->T;
      /* tones with zero frequency are constant along t: sum them once */
      double dc_r = 0.0, dc_i = 0.0;
      for (int k = 0; k < j->n_tones; ++k) {
        if (j->freq[k] != 0.0) continue;
        double ph = j->phase[k * j->n_in + i] + j->slope[k * j->n_in + i] * (double)c;
        dc_r += j->amp[k] * cos(ph);
        dc_i += j->amp[k] * sin(ph);
      }
      for (int t = 0; t < j->T; ++t) {
        uint64_t ta = j->block * (uint64_t)j->T + (uint64_t)t;
        uint32_t x[4] = {(uint32_t)ta, (uint32_t)(ta >> 32), (uint32_t)i, (uint32_t)c};
        synth_philox4x32_10(x, key);
        double u1 = ((double)(x[0] >> 5) * 67108864.0 + (double)(x[1] >> 6) + 1.0) * inv53;
        double u2 = ((double)(x[2] >> 5) * 67108864.0 + (double)(x[3] >> 6)) * inv53;
        double rad = j->sigma * sqrt(-2.0 * log(u1));
        double zr = rad * cos(two_pi * u2) + dc_r, zi = rad * sin(two_pi * u2) + dc_i;
        for (int k = 0; k < j->n_tones; ++k) {
          if (j->freq[k] == 0.0) continue;
          double ph = two_pi * j->freq[k] * (double)ta + j->phase[k * j->n_in + i] +
                      j->slope[k * j->n_in + i] * (double)c;
          zr += j->amp[k] * cos(ph);
          zi += j->amp[k] * sin(ph);
        }
        int re = clip7(zr), im = clip7(zi);
        row[t] = (uint8_t)(((re & 15) << 4) | (im & 15));
      }
    }
  }
  return NULL;
}

/*
 * Writes out[n_chan][n_in][T] (one byte per complex sample) for channels
 * c0 .. c0+n_chan-1 of block `block`.  phase and slope are [n_tones][n_in]
 * arrays (radians, radians per channel).  Returns 0, or -1 on bad sizes.
 */
int synth_block(uint8_t *out, int n_in, int n_chan, int T, int c0, uint64_t seed,
                uint64_t block, double sigma, int n_tones, const double *amp,
                const double *freq, const double *phase, const double *slope,
                int n_threads) {
  if (!out || n_in <= 0 || n_chan <= 0 || T <= 0 || n_tones < 0) return -1;
  if (n_tones > 0 && (!amp || !freq || !phase || !slope)) return -1;
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_chan) n_threads = n_chan;
  job_t *jobs = (job_t *)calloc((size_t)n_threads, sizeof(job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -1; }
  for (int k = 0; k < n_threads; ++k) {
    job_t *j = &jobs[k];
    j->out = out; j->n_in = n_in; j->n_chan = n_chan; j->T = T; j->c0 = c0;
    j->chan_lo = (int)((long long)n_chan * k / n_threads);
    j->chan_hi = (int)((long long)n_chan * (k + 1) / n_threads);
    j->seed = seed; j->block = block; j->sigma = sigma; j->n_tones = n_tones;
    j->amp = amp; j->freq = freq; j->phase = phase; j->slope = slope;
  }
  int started = 0;
  for (int k = 1; k < n_threads; ++k) {
    if (pthread_create(&th[k], NULL, work, &jobs[k]) != 0) break;
    started = k;
  }
  work(&jobs[0]);
  for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
  /* any job whose thread failed to start runs here */
  for (int k = started + 1; k < n_threads; ++k) work(&jobs[k]);
  free(jobs); free(th);
  return 0;
}
