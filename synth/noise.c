/* Seeded synthetic inputs for stochastic texture filtering workloads.
 *
 * This module only MAKES inputs: value-noise textures and grids, a cloud-like
 * sparse occupancy, and pinhole-camera ray-march sample positions.  It holds no
 * part of the filtering method, and both the CUDA library's tests and the oracle
 * read the same arrays it writes.
 *
 * Value noise: pseudo-random lattice values in [0,1) from an integer hash of the
 * lattice point and a seed, blended with the quintic fade 6t^5 - 15t^4 + 10t^3;
 * fractal (fBm) sums of octaves with lacunarity 2 and a given gain, divided by the
 * sum of the octave amplitudes.  The integer hash is Wellons' "lowbias32".
 *
 * Plain C99 + OpenMP; compiled with -ffp-contract=off so that x86-64 and aarch64
 * hosts produce the same floats.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

static inline uint32_t hash4(uint32_t a, uint32_t b, uint32_t c, uint32_t seed) {
  uint32_t h = hash32(seed ^ 0x68bc21ebU);
  h = hash32(h ^ a);
  h = hash32(h ^ b);
  h = hash32(h ^ c);
  return h;
}

static inline double lattice(int64_t x, int64_t y, int64_t z, uint32_t seed) {
  return (double)(hash4((uint32_t)x, (uint32_t)y, (uint32_t)z, seed) >> 8) * (1.0 / 16777216.0);
}

static inline double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }

static double value_noise3(double x, double y, double z, uint32_t seed) {
  double fx = floor(x), fy = floor(y), fz = floor(z);
  int64_t ix = (int64_t)fx, iy = (int64_t)fy, iz = (int64_t)fz;
  double tx = fade(x - fx), ty = fade(y - fy), tz = fade(z - fz);
  double c[2][2][2];
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 2; ++i) c[k][j][i] = lattice(ix + i, iy + j, iz + k, seed);
  double r[2];
  for (int k = 0; k < 2; ++k) {
    double a = c[k][0][0] + (c[k][0][1] - c[k][0][0]) * tx;
    double b = c[k][1][0] + (c[k][1][1] - c[k][1][0]) * tx;
    r[k] = a + (b - a) * ty;
  }
  return r[0] + (r[1] - r[0]) * tz;
}

static double fbm3(double x, double y, double z, uint32_t seed, int octaves, double gain) {
  double sum = 0.0, amp = 1.0, norm = 0.0, f = 1.0;
  for (int o = 0; o < octaves; ++o) {
    sum += amp * value_noise3(x * f, y * f, z * f, seed + 1013u * (uint32_t)o);
    norm += amp;
    amp *= gain;
    f *= 2.0;
  }
  return sum / norm;
}

/* 2D image, out[(y*W + x)*C + c]; texel centres at (x + 1/2, y + 1/2); each channel
 * is normalised to [0, 1] by its own minimum and maximum. */
void synth_fbm2_image(uint32_t seed, int W, int H, int C, double period, int octaves,
                      double gain, float* out) {
  const int64_t n = (int64_t)W * H;
  double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
  for (int c = 0; c < C; ++c) {
    uint32_t s = seed * 7919u + 104729u * (uint32_t)c;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      int64_t x = i % W, y = i / W;
      tmp[i] = fbm3((x + 0.5) / period, (y + 0.5) / period, 0.5, s, octaves, gain);
    }
    double lo = tmp[0], hi = tmp[0];
    for (int64_t i = 1; i < n; ++i) {
      if (tmp[i] < lo) lo = tmp[i];
      if (tmp[i] > hi) hi = tmp[i];
    }
    double inv = hi > lo ? 1.0 / (hi - lo) : 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i * C + c] = (float)((tmp[i] - lo) * inv);
  }
  free(tmp);
}

/* 3D grid of fBm values in [0, 1), out[(z*ny + y)*nx + x], sampled at integer
 * positions offset by (ox, oy, oz), divided by period. */
void synth_fbm3_grid(uint32_t seed, int nx, int ny, int nz, int64_t ox, int64_t oy, int64_t oz,
                     double period, int octaves, double gain, float* out) {
  const int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t x = i % nx, y = (i / nx) % ny, z = i / ((int64_t)nx * ny);
    out[i] = (float)fbm3((x + ox + 0.5) / period, (y + oy + 0.5) / period,
                         (z + oz + 0.5) / period, seed, octaves, gain);
  }
}

/* Cloud-like field on a coarse cell grid of size n^3 (each cell one sparse leaf):
 * fBm times a radial falloff max(0, 1 - r / R) about the domain centre. */
void synth_cloud_cells(uint32_t seed, int n, double period, int octaves, double gain,
                       double radius_frac, float* out) {
  const int64_t total = (int64_t)n * n * n;
  const double c = 0.5 * n, R = radius_frac * n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < total; ++i) {
    int64_t x = i % n, y = (i / n) % n, z = i / ((int64_t)n * n);
    double dx = x + 0.5 - c, dy = (y + 0.5 - c) * 1.6, dz = z + 0.5 - c;
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double fall = 1.0 - r / R;
    if (fall < 0.0) fall = 0.0;
    out[i] = (float)(fbm3((x + 0.5) / period, (y + 0.5) / period, (z + 0.5) / period, seed,
                          octaves, gain) * fall);
  }
}

/* Voxel values of active 8^3 leaves, out[leaf][x][y][z] (512 per leaf): a fine fBm
 * density in (0, 1]. */
void synth_leaf_values(uint32_t seed, int64_t n_leaves, const int32_t* origins, double period,
                       int octaves, double gain, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < n_leaves; ++l) {
    const int32_t ox = origins[3 * l], oy = origins[3 * l + 1], oz = origins[3 * l + 2];
    float* dst = out + 512 * l;
    for (int x = 0; x < 8; ++x)
      for (int y = 0; y < 8; ++y)
        for (int z = 0; z < 8; ++z) {
          double v = fbm3((ox + x + 0.5) / period, (oy + y + 0.5) / period,
                          (oz + z + 0.5) / period, seed, octaves, gain);
          dst[(x << 6) | (y << 3) | z] = (float)(0.05 + 0.95 * v);
        }
  }
}

/* Pinhole camera on a sphere around `centre`, looking at the centre, vertical field
 * of view `fov_deg`; each of the W*H rays takes `steps` samples at distances
 * radius - half_span + (s + j) * 2 * half_span / steps, j a per-sample hash jitter in
 * [0, 1).  Output float32 xyz in ray-major, step-minor order:
 * out[((py*W + px)*steps + s)*3 + k]. */
void synth_camera_queries(uint32_t seed, int W, int H, int steps, const double* centre,
                          double radius, const double* view_dir, double fov_deg,
                          double half_span, float* out) {
  double d[3] = {view_dir[0], view_dir[1], view_dir[2]};
  double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int k = 0; k < 3; ++k) d[k] /= dl;
  double cam[3] = {centre[0] - radius * d[0], centre[1] - radius * d[1], centre[2] - radius * d[2]};
  double up[3] = {0.0, 0.0, 1.0};
  if (fabs(d[2]) > 0.99) { up[0] = 0.0; up[1] = 1.0; up[2] = 0.0; }
  double rt[3] = {d[1] * up[2] - d[2] * up[1], d[2] * up[0] - d[0] * up[2], d[0] * up[1] - d[1] * up[0]};
  double rl = sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
  for (int k = 0; k < 3; ++k) rt[k] /= rl;
  double uu[3] = {rt[1] * d[2] - rt[2] * d[1], rt[2] * d[0] - rt[0] * d[2], rt[0] * d[1] - rt[1] * d[0]};
  const double th = tan(0.5 * fov_deg * 3.14159265358979323846 / 180.0);
  const double aspect = (double)W / (double)H;
  const int64_t rays = (int64_t)W * H;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < rays; ++r) {
    const int px = (int)(r % W), py = (int)(r / W);
    double sx = (2.0 * (px + 0.5) / W - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * (py + 0.5) / H) * th;
    double dir[3];
    for (int k = 0; k < 3; ++k) dir[k] = d[k] + sx * rt[k] + sy * uu[k];
    double len = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int k = 0; k < 3; ++k) dir[k] /= len;
    for (int s = 0; s < steps; ++s) {
      double j = (double)(hash4((uint32_t)r, (uint32_t)s, 0x51ed27u, seed) >> 8) * (1.0 / 16777216.0);
      double t = radius - half_span + (s + j) * (2.0 * half_span / steps);
      float* o = out + 3 * (r * steps + s);
      for (int k = 0; k < 3; ++k) o[k] = (float)(cam[k] + t * dir[k]);
    }
  }
}

/* Uniform float32 values in [0, 1) from the hash, out[i] for i in [0, n): used for
 * query coordinates and footprints so that large batches are generated quickly. */
void synth_uniform(uint32_t seed, uint32_t stream, int64_t n, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    uint32_t h = hash4((uint32_t)i, (uint32_t)((uint64_t)i >> 32), stream, seed);
    out[i] = (float)((double)(h >> 8) * (1.0 / 16777216.0));
  }
}
