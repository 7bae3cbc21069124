/*
 * FP64 CPU oracle for the 3D complex-to-complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * source, header, table or helper with the CUDA path.
 *
 * What it computes (the paper, section "Approach", Eq. 1):
 *
 *   F(kx,ky,kz) = sum_z sum_y sum_x f(x,y,z) W_nx^(x kx) W_ny^(y ky) W_nz^(z kz),
 *   W_n = exp(s * 2 pi i / n),   s = -1 forward, s = +1 inverse (unnormalised).
 *
 * Eq. 1 prints the per-axis roots as W_x, W_y, W_z while the text defines a
 * single W_N; the reading used here is W_n = exp(-2 pi i / n) with n the
 * length of that axis (all equal for the cubic grids).
 *
 * oracle_dft3d follows the decomposition stated right after Eq. 1: a 1D
 * transform along x, then along y, then along z.  Each 1D transform is the
 * plain O(n^2) definition  out[k] = sum_j in[j] * T[(j*k) mod n]  with
 * T[m] = (cos(2 pi m/n), s*sin(2 pi m/n)) evaluated in double precision by
 * this file.  No FFT factorisation, no blocking.
 *
 * oracle_dft3d_brute is the literal triple sum of Eq. 1 (n^6 terms), each
 * term's phase formed from the full exponent; it exists to pin the separable
 * form.
 *
 * Layout: interleaved complex128 (re, im), index ((b*nz + z)*ny + y)*nx + x,
 * x fastest.  Returns 0 on success, -1 on invalid arguments, -2 on
 * allocation failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORACLE_TWO_PI = 6.283185307179586476925286766559;

/* Roots of unity of order n: T[m] = exp(s*2*pi*i*m/n), m in [0, n). */
static double* make_roots(int n, int sign) {
  double* t = (double*)malloc(sizeof(double) * 2 * (size_t)n);
  if (!t) return NULL;
  for (int m = 0; m < n; ++m) {
    double a = ORACLE_TWO_PI * (double)m / (double)n;
    t[2 * m] = cos(a);
    t[2 * m + 1] = (double)sign * sin(a);
  }
  return t;
}

/*
 * One axis of the separable transform.  The grid is viewed as
 * [outer][n][inner] complex values; every (outer, inner) line of length n is
 * transformed by the direct definition.
 */
static void dft_axis(const double* in, double* out, int64_t outer, int n,
                     int64_t inner, const double* T) {
  const int64_t lines = outer * inner;
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < lines; ++l) {
    const int64_t o = l / inner, i = l % inner;
    const double* src = in + 2 * (o * n * inner + i);
    double* dst = out + 2 * (o * n * inner + i);
    for (int k = 0; k < n; ++k) {
      double re = 0.0, im = 0.0;
      int m = 0; /* (j*k) mod n, advanced by k per step of j */
      for (int j = 0; j < n; ++j, m = (m + k >= n) ? m + k - n : m + k) {
        const double wr = T[2 * m], wi = T[2 * m + 1];
        const double xr = src[2 * (int64_t)j * inner];
        const double xi = src[2 * (int64_t)j * inner + 1];
        re += xr * wr - xi * wi;
        im += xr * wi + xi * wr;
      }
      dst[2 * (int64_t)k * inner] = re;
      dst[2 * (int64_t)k * inner + 1] = im;
    }
  }
}

int oracle_dft3d(const double* in, double* out, int nx, int ny, int nz,
                 int batch, int sign) {
  if (!in || !out || nx < 1 || ny < 1 || nz < 1 || batch < 0) return -1;
  if (sign != -1 && sign != 1) return -1;
  if (batch == 0) return 0;
  const int64_t pts = (int64_t)nx * ny * nz;
  const int64_t total = pts * batch;
  double* tmp = (double*)malloc(sizeof(double) * 2 * (size_t)total);
  double* tx = make_roots(nx, sign);
  double* ty = make_roots(ny, sign);
  double* tz = make_roots(nz, sign);
  if (!tmp || !tx || !ty || !tz) {
    free(tmp); free(tx); free(ty); free(tz);
    return -2;
  }
  /* x: lines of length nx, contiguous.  in -> out */
  dft_axis(in, out, total / nx, nx, 1, tx);
  /* y: [b*nz][ny][nx].  out -> tmp */
  dft_axis(out, tmp, (int64_t)batch * nz, ny, nx, ty);
  /* z: [b][nz][ny*nx].  tmp -> out */
  dft_axis(tmp, out, batch, nz, (int64_t)ny * nx, tz);
  free(tmp); free(tx); free(ty); free(tz);
  return 0;
}

/*
 * Literal Eq. 1: every output is the full triple sum with the phase of each
 * term computed from the reduced combined exponent
 *   theta = 2 pi * ( (x kx mod nx)/nx + (y ky mod ny)/ny + (z kz mod nz)/nz ).
 * O((nx ny nz)^2); meant for grids of at most a few hundred points.
 */
int oracle_dft3d_brute(const double* in, double* out, int nx, int ny, int nz,
                       int sign) {
  if (!in || !out || nx < 1 || ny < 1 || nz < 1) return -1;
  if (sign != -1 && sign != 1) return -1;
  const int64_t pts = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < pts; ++k) {
    const int kx = (int)(k % nx), ky = (int)((k / nx) % ny),
              kz = (int)(k / ((int64_t)nx * ny));
    double re = 0.0, im = 0.0;
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const double frac = (double)((x * kx) % nx) / nx +
                              (double)((y * ky) % ny) / ny +
                              (double)((z * kz) % nz) / nz;
          const double th = (double)sign * ORACLE_TWO_PI * frac;
          const double c = cos(th), s = sin(th);
          const int64_t j = ((int64_t)z * ny + y) * nx + x;
          const double xr = in[2 * j], xi = in[2 * j + 1];
          re += xr * c - xi * s;
          im += xr * s + xi * c;
        }
    out[2 * k] = re;
    out[2 * k + 1] = im;
  }
  return 0;
}

/*
 * Selected outputs of Eq. 1 for one grid, one by one: for each requested
 * (kz, ky, kx) the sums over x, then y, then z of the definition,
 *   F = sum_z W_nz^(z kz) sum_y W_ny^(y ky) sum_x W_nx^(x kx) f(x, y, z),
 * each root taken from the reduced exponent (x kx mod nx, ...).  O(nx ny nz)
 * per output, for checking single outputs of grids too large for
 * oracle_dft3d.  points: npts triples (kz, ky, kx); out: npts complex.
 */
int oracle_dft3d_points(const double* in, int nx, int ny, int nz, const int* points, int npts,
                        int sign, double* out) {
  if (!in || !points || !out || nx < 1 || ny < 1 || nz < 1 || npts < 0) return -1;
  if (sign != -1 && sign != 1) return -1;
  double* tx = make_roots(nx, sign);
  double* ty = make_roots(ny, sign);
  double* tz = make_roots(nz, sign);
  if (!tx || !ty || !tz) {
    free(tx); free(ty); free(tz);
    return -2;
  }
  for (int p = 0; p < npts; ++p) {
    const int kz = points[3 * p], ky = points[3 * p + 1], kx = points[3 * p + 2];
    if (kz < 0 || kz >= nz || ky < 0 || ky >= ny || kx < 0 || kx >= nx) {
      free(tx); free(ty); free(tz);
      return -1;
    }
    double re = 0.0, im = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : re, im)
    for (int z = 0; z < nz; ++z) {
      double zr = 0.0, zi = 0.0;  /* sum over y of (sum over x) W^(y ky) */
      for (int y = 0; y < ny; ++y) {
        const double* row = in + 2 * (((int64_t)z * ny + y) * nx);
        double xr = 0.0, xi = 0.0;
        for (int x = 0; x < nx; ++x) {
          const int m = (int)(((int64_t)x * kx) % nx);
          const double wr = tx[2 * m], wi = tx[2 * m + 1];
          xr += row[2 * x] * wr - row[2 * x + 1] * wi;
          xi += row[2 * x] * wi + row[2 * x + 1] * wr;
        }
        const int my = (int)(((int64_t)y * ky) % ny);
        zr += xr * ty[2 * my] - xi * ty[2 * my + 1];
        zi += xr * ty[2 * my + 1] + xi * ty[2 * my];
      }
      const int mz = (int)(((int64_t)z * kz) % nz);
      re += zr * tz[2 * mz] - zi * tz[2 * mz + 1];
      im += zr * tz[2 * mz + 1] + zi * tz[2 * mz];
    }
    out[2 * p] = re;
    out[2 * p + 1] = im;
  }
  free(tx); free(ty); free(tz);
  return 0;
}

/* Threads the OpenMP runtime will use for the parallel loops above. */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
