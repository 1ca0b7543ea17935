// Reductions and the energy spectrum of the velocity field.
//
// Spectrum (Sec. "Turbulence": E(k) is the shell density of 1/2 |v(k)|^2): with
// z = v_x + i v_y, |V_x(k)|^2 + |V_y(k)|^2 = (|Z(k)|^2 + |Z(-k)|^2) / 2, and every shell
// round(|k|) = n is closed under k -> -k, so the shell sum of |V_x|^2 + |V_y|^2 equals the
// shell sum of |Z|^2: one complex 2-D transform serves both components.  The
// transform is a mixed-radix Stockham FFT (radices 2-8 in registers, any larger prime
// factor as a direct DFT stage), rows then a tiled transpose then rows, FP64.
#include "rlbm_device.cuh"
#include "rlbm_launch.h"
#include "rlbm_tma.cuh"

namespace rlbm {

// ---------------------------------------------------------------------------
// Deterministic sum of per-block partials: thread t sums blocks t, t+256, ... in
// order, then thread 0 adds the 256 thread sums in order.
// ---------------------------------------------------------------------------
__global__ void reduce_partials_kernel(const double *__restrict__ partials, long long nblocks,
                                       double *__restrict__ totals) {
  __shared__ double s[4][256];
  const int t = threadIdx.x;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long i = t; i < nblocks; i += 256)
    for (int k = 0; k < 4; ++k) a[k] += partials[i * 4 + k];
  for (int k = 0; k < 4; ++k) s[k][t] = a[k];
  __syncthreads();
  if (t < 4) {
    double v = 0.0;
    for (int i = 0; i < 256; ++i) v += s[t][i];
    totals[t] = v;
  }
}

__global__ void counter_inc_kernel(long long *c, int *tile_ctr) {
  *c += 1;
  *tile_ctr = 0;
}

// Advances the batch step counter between two batched step launches (stream order) and
// clears the tile counter for the next launch.
cudaError_t launch_counter_inc(long long *counter, int *tile_ctr, cudaStream_t st) {
  counter_inc_kernel<<<1, 1, 0, st>>>(counter, tile_ctr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Self-test of the failure path of the bounded waits: one thread waits on an mbarrier that
// nothing arrives on, with the bounded wait the step kernels use on their TMA copies; when
// it runs out after max_cycles SM clocks the timeout is latched in the error word, as a
// step kernel does.  No copy is in flight, so the thread returns at once.
// ---------------------------------------------------------------------------
__global__ void wait_selftest_kernel(unsigned *err, long long max_cycles) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0, max_cycles)) atomicOr(err, ERR_TIMEOUT);
}

cudaError_t launch_wait_selftest(unsigned *err, long long max_cycles, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(err, max_cycles);
  return cudaGetLastError();
}

// Column means of the velocity v = u / u^0 of the moments fields (solid cells hold u = 0):
// j_x(x) = (1/ny) sum_y v^x, j_y likewise.  One block per column, fixed-order sums.
__global__ void column_means_kernel(const double *__restrict__ ux, const double *__restrict__ uy, int nx, int ny,
                                    double *__restrict__ jx, double *__restrict__ jy) {
  const int x = blockIdx.x;
  double ax = 0.0, ay = 0.0;
  for (int y = threadIdx.x; y < ny; y += blockDim.x) {
    const double a = ux[(long long)y * nx + x], b = uy[(long long)y * nx + x];
    const double iu0 = 1.0 / sqrt(1.0 + a * a + b * b);
    ax += a * iu0;
    ay += b * iu0;
  }
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    ax += __shfl_down_sync(0xffffffffu, ax, off);
    ay += __shfl_down_sync(0xffffffffu, ay, off);
  }
  if (lane == 0) { red[0][warp] = ax; red[1][warp] = ay; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0.0, sy = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sx += red[0][w]; sy += red[1][w]; }
    jx[x] = sx / ny;
    jy[x] = sy / ny;
  }
}

cudaError_t launch_column_means(const double *ux, const double *uy, int nx, int ny, double *jx, double *jy,
                                cudaStream_t st) {
  column_means_kernel<<<nx, 256, 0, st>>>(ux, uy, nx, ny, jx, jy);
  return cudaGetLastError();
}

// Halo rows of a strip: block p copies the padded row of plane p between the population
// buffer and the message buffer, 16 bytes per thread and step (rows start on 128-byte lines
// of the buffer; the message buffer is 16-byte aligned).
__global__ void halo_copy_kernel(char *__restrict__ pop, const HaloRows rows, long long row_bytes,
                                 char *__restrict__ buf, bool pack) {
  const int p = blockIdx.x;
  uint4 *a = reinterpret_cast<uint4 *>(pop + rows.off[p]);
  uint4 *b = reinterpret_cast<uint4 *>(buf + p * row_bytes);
  const long long n = row_bytes / 16;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    if (pack) b[i] = a[i];
    else a[i] = b[i];
  }
}

cudaError_t launch_halo_copy(char *pop, const HaloRows &rows, long long row_bytes, char *buf, bool pack,
                             cudaStream_t st) {
  if (rows.nplanes < 1) return cudaSuccess;
  halo_copy_kernel<<<rows.nplanes, 256, 0, st>>>(pop, rows, row_bytes, buf, pack);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *partials, long long nblocks, double *totals, cudaStream_t st) {
  reduce_partials_kernel<<<1, 256, 0, st>>>(partials, nblocks, totals);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FFT
// ---------------------------------------------------------------------------
struct FftPlan {
  int n, nstages;
  int radix[40];
};

static FftPlan make_plan(int n) {
  FftPlan p;
  p.n = n;
  p.nstages = 0;
  int m = n;
  const int pref[] = {8, 4, 2, 3, 5, 7};
  for (int r : pref)
    while (m % r == 0 && (r != 8 || m % 8 == 0)) { p.radix[p.nstages++] = r; m /= r; }
  for (int f = 11; m > 1; f += 2)
    while (m % f == 0) { p.radix[p.nstages++] = f; m /= f; }
  return p;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// DFT of length 4 (W = exp(-+2 pi i / 4) from the twiddle table, W^2 = -1) by two levels of
// sums and differences: X_0 = a0 + a2, X_1 = a1 + a3, X_2 = a0 - a2, X_3 = a1 - a3.
__device__ __forceinline__ void dft4(double2 v0, double2 v1, double2 v2, double2 v3, double2 W, double2 X[4]) {
  const double2 a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = cmul(csub(v1, v3), W);
  X[0] = cadd(a0, a2);
  X[1] = cadd(a1, a3);
  X[2] = csub(a0, a2);
  X[3] = csub(a1, a3);
}

// One block transforms one row of length n in place (ping-pong between a and b);
// tw[t] = exp(-2 pi i t / n).  Stage with radix R after radices of product Ns:
//   v_r = x[j + r n/R] * w^(r (j mod Ns) n/(Ns R)),  y[(j div Ns) Ns R + (j mod Ns) + k Ns] = DFT_R(v)_k.
// Radices 2, 4 and 8 use their butterflies (8 = two length-4 transforms of the even and
// odd inputs joined by W_8^k); the others evaluate the length-R sums directly (O(n R) work
// for the stage; a prime factor above 8 shares its outputs over the block's threads).
__global__ void fft_rows_kernel(double2 *a, double2 *b, const double2 *__restrict__ tw,
                                FftPlan plan) {
  const int n = plan.n;
  double2 *src = a + (long long)blockIdx.x * n;
  double2 *dst = b + (long long)blockIdx.x * n;
  int Ns = 1;
  for (int s = 0; s < plan.nstages; ++s) {
    const int R = plan.radix[s];
    const int nR = n / R;
    const int stride = n / (Ns * R);
    if (R > 8) {
      // a prime factor above 8: direct sums of length R, one output (j, k) per thread, so a
      // prime length (nR = 1) spreads over the block instead of falling to one thread
      for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int j = t / R, k = t - j * R;
        const int jm = j % Ns;
        const int base = (j / Ns) * Ns * R + jm;
        double2 acc = make_double2(0.0, 0.0);
        for (int r = 0; r < R; ++r) {
          const double2 v = cmul(src[j + r * nR], tw[r * jm * stride]);
          const double2 e = tw[((r * k) % R) * nR];
          acc.x += v.x * e.x - v.y * e.y;
          acc.y += v.x * e.y + v.y * e.x;
        }
        dst[base + k * Ns] = acc;
      }
      __syncthreads();
      double2 *tmp = src; src = dst; dst = tmp;
      Ns *= R;
      continue;
    }
    for (int j = threadIdx.x; j < nR; j += blockDim.x) {
      const int jm = j % Ns;
      const int base = (j / Ns) * Ns * R + jm;
      if (R == 2 || R == 4 || R == 8) {
        double2 v[8];
        for (int r = 0; r < R; ++r) v[r] = cmul(src[j + r * nR], tw[r * jm * stride]);  // r jm stride < n
        if (R == 2) {
          dst[base] = cadd(v[0], v[1]);
          dst[base + Ns] = csub(v[0], v[1]);
        } else if (R == 4) {
          double2 X[4];
          dft4(v[0], v[1], v[2], v[3], tw[nR], X);
          for (int k = 0; k < 4; ++k) dst[base + k * Ns] = X[k];
        } else {
          double2 E[4], O[4];
          const double2 W4 = tw[2 * nR];  // W_8^2
          dft4(v[0], v[2], v[4], v[6], W4, E);
          dft4(v[1], v[3], v[5], v[7], W4, O);
          for (int k = 0; k < 4; ++k) {
            const double2 t = k == 0 ? O[0] : cmul(O[k], tw[k * nR]);  // W_8^k O_k
            dst[base + k * Ns] = cadd(E[k], t);
            dst[base + (k + 4) * Ns] = csub(E[k], t);
          }
        }
      } else {  // radix 3, 5 or 7: the length-R sums
        double2 v[8];
        for (int r = 0; r < R; ++r) v[r] = cmul(src[j + r * nR], tw[r * jm * stride]);  // r jm stride < n
        for (int k = 0; k < R; ++k) {
          double2 acc = v[0];
          for (int r = 1; r < R; ++r) {
            const int t = ((r * k) % R) * nR;
            acc.x += v[r].x * tw[t].x - v[r].y * tw[t].y;
            acc.y += v[r].x * tw[t].y + v[r].y * tw[t].x;
          }
          dst[base + k * Ns] = acc;
        }
      }
    }
    __syncthreads();
    double2 *tmp = src; src = dst; dst = tmp;
    Ns *= R;
  }
}

__global__ void make_z_kernel(const double *__restrict__ ux, const double *__restrict__ uy, double2 *__restrict__ z,
                              long long ncell) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const double a = ux[c], b = uy[c];
  const double u0 = sqrt(1.0 + a * a + b * b);
  z[c] = make_double2(a / u0, b / u0);
}

// out[x * ny + y] = in[y * nx + x]
__global__ void transpose_kernel(const double2 *__restrict__ in, double2 *__restrict__ out, int nx, int ny) {
  __shared__ double2 tile[32][33];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int x = x0 + threadIdx.x, y = y0 + k;
    if (x < nx && y < ny) tile[k][threadIdx.x] = in[(long long)y * nx + x];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int y = y0 + threadIdx.x, x = x0 + k;
    if (x < nx && y < ny) out[(long long)x * ny + y] = tile[threadIdx.x][k];
  }
}

// Z is transposed: row = k_x index, column = k_y index.  E[round|k|] += 1/2 |Z|^2 / (nx ny)^2.
__global__ void bin_kernel(const double2 *__restrict__ Z, int nx, int ny, double *__restrict__ bins, int nbins,
                           double scale) {
  extern __shared__ double sb[];
  const bool use_smem = nbins <= 6144;
  if (use_smem)
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) sb[i] = 0.0;
  __syncthreads();
  const int qx = blockIdx.x;
  const int kx = qx < (nx + 1) / 2 ? qx : qx - nx;
  for (int qy = threadIdx.x; qy < ny; qy += blockDim.x) {
    const int ky = qy < (ny + 1) / 2 ? qy : qy - ny;
    const int n = __double2int_rn(sqrt((double)kx * kx + (double)ky * ky));
    if (n >= nbins) continue;
    const double2 v = Z[(long long)qx * ny + qy];
    const double e = scale * (v.x * v.x + v.y * v.y);
    if (use_smem) atomicAdd(&sb[n], e);
    else atomicAdd(&bins[n], e);
  }
  __syncthreads();
  if (use_smem)
    for (int i = threadIdx.x; i < nbins; i += blockDim.x)
      if (sb[i] != 0.0) atomicAdd(&bins[i], sb[i]);
}

// Z = 2-D transform of v_x + i v_y (v = u / u^0), laid out [k_x][k_y]; returns which of
// the two work buffers holds it.
static double2 *velocity_transform(const double *ux, const double *uy, int nx, int ny, const double2 *twx,
                                   const double2 *twy, double2 *z0, double2 *z1, cudaStream_t st) {
  const long long ncell = (long long)nx * ny;
  make_z_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(ux, uy, z0, ncell);
  const FftPlan px = make_plan(nx), py = make_plan(ny);
  fft_rows_kernel<<<ny, 256, 0, st>>>(z0, z1, twx, px);
  double2 *r = (px.nstages % 2) ? z1 : z0;  // result of the row transforms
  double2 *o = (px.nstages % 2) ? z0 : z1;
  transpose_kernel<<<dim3((nx + 31) / 32, (ny + 31) / 32), dim3(32, 8), 0, st>>>(r, o, nx, ny);
  fft_rows_kernel<<<nx, 256, 0, st>>>(o, r, twy, py);
  return (py.nstages % 2) ? r : o;
}

// Energy of a band of wave vectors, k2lo <= k_x^2 + k_y^2 < k2hi (k2hi <= 0: no upper
// bound): (1/2) sum |V_x|^2 + |V_y|^2 / (nx ny)^2, as the spectrum's bins but with an exact
// integer band edge (the velocity filter that removes the driven range).  One FP64 partial
// per block (k_x column), summed in order afterwards.
__global__ void band_kernel(const double2 *__restrict__ Z, int nx, int ny, long long k2lo, long long k2hi,
                            double scale, double *__restrict__ partials) {
  const int qx = blockIdx.x;
  const long long kx = qx < (nx + 1) / 2 ? qx : qx - nx;
  double acc = 0.0;
  for (int qy = threadIdx.x; qy < ny; qy += blockDim.x) {
    const long long ky = qy < (ny + 1) / 2 ? qy : qy - ny;
    const long long k2 = kx * kx + ky * ky;
    if (k2 < k2lo || (k2hi > 0 && k2 >= k2hi)) continue;
    const double2 v = Z[(long long)qx * ny + qy];
    acc += scale * (v.x * v.x + v.y * v.y);
  }
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partials[(long long)qx * 4] = s;
    partials[(long long)qx * 4 + 1] = partials[(long long)qx * 4 + 2] = partials[(long long)qx * 4 + 3] = 0.0;
  }
}

cudaError_t launch_band_energy(const double *ux, const double *uy, int nx, int ny, const double2 *twx,
                               const double2 *twy, double2 *z0, double2 *z1, long long k2lo, long long k2hi,
                               double *partials, double *out4, cudaStream_t st) {
  double2 *Z = velocity_transform(ux, uy, nx, ny, twx, twy, z0, z1, st);
  const double scale = 0.5 / ((double)nx * ny * (double)nx * ny);
  band_kernel<<<nx, 256, 0, st>>>(Z, nx, ny, k2lo, k2hi, scale, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(partials, nx, out4, st);
}

cudaError_t launch_spectrum(const double *ux, const double *uy, int nx, int ny, const double2 *twx,
                            const double2 *twy, double2 *z0, double2 *z1, double *bins, int nbins,
                            cudaStream_t st) {
  const long long ncell = (long long)nx * ny;
  double2 *Z = velocity_transform(ux, uy, nx, ny, twx, twy, z0, z1, st);
  cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(double) * nbins, st);
  if (e != cudaSuccess) return e;
  const size_t smem = nbins <= 6144 ? sizeof(double) * nbins : 0;
  const double scale = 0.5 / ((double)ncell * (double)ncell);
  bin_kernel<<<nx, 256, smem, st>>>(Z, nx, ny, bins, nbins, scale);
  return cudaGetLastError();
}

}  // namespace rlbm
