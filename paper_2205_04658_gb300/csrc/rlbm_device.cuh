// Device side of the relativistic lattice Boltzmann update (arXiv 2205.04658).
//
// State: normalised deviations h_i = f_i / (w_i eps0) - 1 of the post-collision
// populations f*_i, one SoA plane per folded velocity class, row pitch `pitch`.
//
// The paper's momentum set is the 26 unit vectors along the D3Q27 neighbour
// directions (Part I "Model and Methods"; Sec. "Boltzmann to Lattice Boltzmann").
// On a lattice one node thick in z, every population is even in v_z, so the pair
// (v_x, v_y, +v_z), (v_x, v_y, -v_z) is carried as one class with the summed weight
// and its v_z^2; this folds 26 directions into 17 classes exactly.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace rlbm {

// keep the scalar math overloads visible next to the packed-pair ones defined below
using ::fma;
using ::fmax;

enum : unsigned { ERR_UNSTABLE = 1u, ERR_UNPHYSICAL = 2u, ERR_TIMEOUT = 4u };

// ---------------------------------------------------------------------------
// Velocity classes.  VS = 3: the paper's set folded to 17 in-plane classes
// (weights 1/21, 4/105, 9/280 per 3-D direction, degree-7 spherical rule);
// VS = 2: 8 directions on the unit circle, weights 1/8.
// ---------------------------------------------------------------------------
#define RLBM_S2 0.70710678118654752440
#define RLBM_S3 0.57735026918962576451

template <int VS> struct VSet;

template <> struct VSet<3> {
  static constexpr int Q = 17;
  static constexpr int DP = 3;
  __host__ __device__ static constexpr double vx(int q) {
    return q == 1 ? 1.0 : q == 3 ? -1.0
         : (q == 5 || q == 8 || q == 9) ? RLBM_S2 : (q == 6 || q == 7 || q == 11) ? -RLBM_S2
         : (q == 13 || q == 16) ? RLBM_S3 : (q == 14 || q == 15) ? -RLBM_S3 : 0.0;
  }
  __host__ __device__ static constexpr double vy(int q) {
    return q == 2 ? 1.0 : q == 4 ? -1.0
         : (q == 5 || q == 6 || q == 10) ? RLBM_S2 : (q == 7 || q == 8 || q == 12) ? -RLBM_S2
         : (q == 13 || q == 14) ? RLBM_S3 : (q == 15 || q == 16) ? -RLBM_S3 : 0.0;
  }
  __host__ __device__ static constexpr double vz2(int q) {
    return q == 0 ? 1.0 : (q >= 9 && q <= 12) ? 0.5 : (q >= 13) ? (1.0 / 3.0) : 0.0;
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 2.0 / 21.0 : q <= 4 ? 1.0 / 21.0 : q <= 8 ? 4.0 / 105.0
         : q <= 12 ? 8.0 / 105.0 : 9.0 / 140.0;
  }
  __host__ __device__ static constexpr int opp(int q) {
    return q == 0 ? 0 : q <= 4 ? ((q - 1 + 2) % 4) + 1 : q <= 8 ? ((q - 5 + 2) % 4) + 5
         : q <= 12 ? ((q - 9 + 2) % 4) + 9 : ((q - 13 + 2) % 4) + 13;
  }
  // f_eq coefficients: h_eq = (eps^ - 1) + CA eps^ u0 (u.v) + CB eps^ (u.v)^2 - CC eps^ |u|^2
  static constexpr double CA = 4.0, CB = 10.0, CC = 2.0;
  static constexpr double TAU_NUM = 5.0;  // tau_R = 5 (eta/s) / T
};

template <> struct VSet<2> {
  static constexpr int Q = 8;
  static constexpr int DP = 2;
  __host__ __device__ static constexpr double vx(int q) {
    return q == 0 ? 1.0 : q == 4 ? -1.0 : (q == 1 || q == 7) ? RLBM_S2 : (q == 3 || q == 5) ? -RLBM_S2 : 0.0;
  }
  __host__ __device__ static constexpr double vy(int q) {
    return q == 2 ? 1.0 : q == 6 ? -1.0 : (q == 1 || q == 3) ? RLBM_S2 : (q == 5 || q == 7) ? -RLBM_S2 : 0.0;
  }
  __host__ __device__ static constexpr double vz2(int) { return 0.0; }
  __host__ __device__ static constexpr double w(int) { return 0.125; }
  __host__ __device__ static constexpr int opp(int q) { return (q + 4) % 8; }
  static constexpr double CA = 3.0, CB = 6.0, CC = 1.5;
  static constexpr double TAU_NUM = 4.0;
};

// sign of the streaming displacement of class q (compile time)
template <int VS> __host__ __device__ constexpr int sgnx(int q) {
  return VSet<VS>::vx(q) > 1e-12 ? 1 : VSet<VS>::vx(q) < -1e-12 ? -1 : 0;
}
template <int VS> __host__ __device__ constexpr int sgny(int q) {
  return VSet<VS>::vy(q) > 1e-12 ? 1 : VSet<VS>::vy(q) < -1e-12 ? -1 : 0;
}

// ---------------------------------------------------------------------------
// Storage conversions
// ---------------------------------------------------------------------------
// Scale of the stored deviations.  FP16 storage holds 2^8 h: the deviations down to 2^-22
// (not 2^-14) then lie in FP16's normal range, where the stochastic rounding of the stores
// is unbiased, and |h| up to 255 stays below FP16's largest value.  Powers of two, so the
// scaling itself is exact.
template <typename S> struct HScale {
  static constexpr float up = 1.0f, down = 1.0f;
};
template <> struct HScale<__half> {
  static constexpr float up = 256.0f, down = 1.0f / 256.0f;
};

// h of one stored value (load_h: global memory through the read-only path; load_h_s:
// shared memory) and h to its stored form.
template <typename S, typename R> __device__ __forceinline__ R load_h(const S *p) { return (R)__ldg(p); }
template <> __device__ __forceinline__ float load_h<__half, float>(const __half *p) {
  return __half2float(__ldg(p)) * HScale<__half>::down;
}
template <> __device__ __forceinline__ float load_h<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
  return __bfloat162float(__ldg(p));
}
template <typename S, typename R> __device__ __forceinline__ R load_h_s(const S *p) { return (R)*p; }
template <> __device__ __forceinline__ float load_h_s<__half, float>(const __half *p) {
  return __half2float(*p) * HScale<__half>::down;
}
template <> __device__ __forceinline__ float load_h_s<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}
// A stored value as FP32 without the storage scale (the paired step kernels fold 1 / up
// into their pull weights).
template <typename S> __device__ __forceinline__ float load_s_raw(const S *p) { return load_h_s<S, float>(p); }
template <> __device__ __forceinline__ float load_s_raw<__half>(const __half *p) { return __half2float(*p); }
template <typename S, typename R> __device__ __forceinline__ S store_h(R v) { return (S)v; }
template <> __device__ __forceinline__ __half store_h<__half, float>(float v) {
  return __float2half_rn(v * HScale<__half>::up);
}
template <> __device__ __forceinline__ __nv_bfloat16 store_h<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

template <typename S> struct RealOf { using type = float; };
template <> struct RealOf<double> { using type = double; };

// ---------------------------------------------------------------------------
// Storage layout.  Each population plane holds (ny + 2) rows of `pitch` elements:
// interior cell (x, y) sits at row y + 1, column x + XOFF; column XOFF - 1 and XOFF + nx
// and rows 0 and ny + 1 are ghost copies of the periodic neighbours (solid walls keep
// zero ghost rows).  XOFF is 128 bytes, so interior rows start on a 128-byte line.
// ---------------------------------------------------------------------------
template <typename S> struct PadLayout {
  static constexpr int XOFF = 128 / (int)sizeof(S);
  static constexpr int V = 16 / (int)sizeof(S);  // TMA x granule (16 bytes)
};

// ---------------------------------------------------------------------------
// Parameters
// ---------------------------------------------------------------------------
template <typename R> struct alignas(16) R4 { R x, y, z, w; };
template <typename R> struct alignas(2 * sizeof(R)) R2 { R x, y; };

template <typename R> struct Geometry {
  int nx, ny, pitch;
  long long plane;          // elements per plane (pitch * (ny + 2))
  int walls;                // y ghost rows are solid (never written)
  const uint16_t *nbmask;   // bit 4: cell solid; bit (dy+1)*3+(dx+1): neighbour (x+dx, y+dy) solid
  R beta[17][4];            // bilinear weights of corners (0,0), (s_x,0), (0,s_y), (s_x,s_y)
  float2 beta2[17][4];      // the same duplicated into pairs (packed two-cell arithmetic)
};

template <typename R> struct Physics {
  R omega0;        // dt T0 / (TAU_NUM eta/s): relaxation factor at eps = eps0
  R fpref;         // -6 dt / T0: force prefactor including dt
  R body_x, body_y;
  R vmax2;         // FP32 path: |v|^2 above which Landau runs in FP64
  int stochastic;  // 16-bit storage: stochastic rounding
  unsigned round_key;
  unsigned step;   // low 32 bits of the step index (rounding bits)
  int y_off;       // lattice row of row 0 (a strip of a larger lattice; else 0): rounding bits
};

// ---------------------------------------------------------------------------
// Stochastic rounding of the 16-bit stores: unbiased (E[round(v)] = v), so the rounding
// errors of successive steps do not add up coherently.  The random bits are a
// counter-based hash of (cell, step, key), advanced by a Weyl step (an odd constant near
// 2^32 / golden ratio added modulo 2^32) per value, so a run repeats exactly.  Every value's
// bits are uniform because the hash is; the 17 values of one cell take evenly spread
// offsets from it.  (An integer add, where a multiplicative generator would occupy the
// FMA pipe that the cell's arithmetic already saturates.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cell_hash(uint32_t x, uint32_t y, uint32_t step, uint32_t key) {
  uint32_t h = (x * 0x9E3779B1u) ^ ((y + 0x7F4A7C15u) * 0x85EBCA77u) ^ ((step ^ key) * 0xC2B2AE3Du);
  h ^= h >> 16; h *= 0x7FEB352Du; h ^= h >> 15; h *= 0x846CA68Bu; h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint32_t next_bits(uint32_t r) { return r + 0x9E3779B9u; }

// v rounded to storage type S: to nearest, or stochastically with the random bits r.
// BF16: adding 16 random bits below the kept mantissa of the FP32 pattern and truncating
// (round toward zero) rounds the magnitude up with probability equal to the dropped
// fraction.  (FP16 pairs: round_pair_f16 below.)
template <typename S> __device__ __forceinline__ S store_round(float v, bool sr, uint32_t r) {
  return store_h<S, float>(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 store_round<__nv_bfloat16>(float v, bool sr, uint32_t r) {
  if (!sr) return __float2bfloat16_rn(v);
  return __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r >> 16)) >> 16));
}

// The two cells of a pair, already multiplied by the storage scale, rounded stochastically
// to FP16 in one packed conversion with the random bits ra, rb (the low half of the result
// holds a, the high half b): 13 random bits are added below the kept FP16 mantissa of each
// FP32 value and the sums are truncated (round toward zero), which rounds the magnitude up
// with probability equal to the dropped fraction.  Below FP16's normal range (2^-14, i.e.
// |h| < 2^-22) the 13 bits do not reach every dropped bit and the rounding leans toward
// zero by less than one FP16 subnormal spacing, 2^-32 in h.
__device__ __forceinline__ uint32_t round_pair_f16_sr(float a, float b, uint32_t ra, uint32_t rb) {
  const float ua = __uint_as_float(__float_as_uint(a) + (ra >> 19));
  const float ub = __uint_as_float(__float_as_uint(b) + (rb >> 19));
  uint32_t d;
  asm("cvt.rz.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(ub), "f"(ua));  // (high, low) = (b, a)
  return d;
}
// The same rounded to nearest.
__device__ __forceinline__ uint32_t round_pair_f16_rn(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

template <typename R> struct Stir {
  int nrows;               // distinct k_y of the shell (0 = no stirring)
  int nmodes;
  const R4<R> *G_cur;      // [nrows][nx]: (Gx.re, Gx.im, Gy.re, Gy.im) of this step
  const R2<R> *EY;         // [nrows][eyp]: exp(i 2 pi k_y(row) y / ny), rows padded to eyp
  int eyp;
  // pipelined preparation of the next steps (done by the same launch)
  R4<R> *G_next;           // [nrows][nx] of step n+1
  const R4<R> *coef_next;  // [nmodes]: (cx.re, cx.im, cy.re, cy.im) of step n+1
  R4<R> *coef_new;         // [nmodes] of step n+2 (written)
  const int *mode_kx;      // [nmodes]
  const int *row_start;    // [nrows+1] mode range of each row (modes sorted by k_y)
  unsigned long long seed;
  long long step_new;      // n + 2
  double amp;
  const double *mode_scale;  // [nmodes] amplitude multipliers sigma_m; NULL = all 1
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the stirring draws
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// Mode m of step n: a = amp sqrt(-2 ln u0) cos(2 pi u1), phi = 2 pi u2, psi = 2 pi u3,
// coefficient pair (cx, cy) = a (cos psi, sin psi) exp(i phi).  FP64.
__device__ inline void stir_draw(unsigned long long seed, long long n, int m, double amp, double out[4]) {
  uint32_t c[4] = {(uint32_t)(n & 0xffffffffll), (uint32_t)m, (uint32_t)((unsigned long long)n >> 32), 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
  double u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) u[j] = ((double)c[j] + 0.5) * 2.3283064365386962890625e-10;
  const double a = amp * sqrt(-2.0 * log(u[0])) * cospi(2.0 * u[1]);
  double sphi, cphi, spsi, cpsi;
  sincospi(2.0 * u[2], &sphi, &cphi);
  sincospi(2.0 * u[3], &spsi, &cpsi);
  out[0] = a * cpsi * cphi; out[1] = a * cpsi * sphi;
  out[2] = a * spsi * cphi; out[3] = a * spsi * sphi;
}

// exp(i pi a) for the stirring phases: FP64 in the FP64 path, FP32 (about 1 ulp) in the
// others.
template <typename R> __device__ __forceinline__ void sincospi_R(R a, R *s, R *c);
template <> __device__ __forceinline__ void sincospi_R<double>(double a, double *s, double *c) { sincospi(a, s, c); }
template <> __device__ __forceinline__ void sincospi_R<float>(float a, float *s, float *c) { sincospif(a, s, c); }

// One entry of the per-row stirring table of a step:
//   G_r(x) = sum_{m in row r} (cx_m, cy_m) exp(i 2 pi k_x,m x / nx),
// the phase evaluated from the exact integer residue k_x,m x mod nx.  The modes of a row
// are summed in four interleaved parts (m = first + l, l + 4, ...), combined as
// (p0 + p1) + (p2 + p3): the table builders that split an entry over four lanes and those
// that do not then give the same bits.  `coef`, `kx` and `row_start` may live in shared
// memory.
template <typename R>
__device__ inline R4<R> stir_entry_part(const R4<R> *coef, const int *kx, const int *row_start, int r, int x, int nx,
                                        int l4) {
  R4<R> g{R(0), R(0), R(0), R(0)};
  const int m1 = row_start[r + 1];
  for (int m = row_start[r] + l4; m < m1; m += 4) {
    int j = (kx[m] * x) % nx;  // |k_x| < nx / 2 and x < nx <= 32768: no 32-bit overflow
    if (j < 0) j += nx;
    R sn, cs;
    sincospi_R<R>(R(2 * j) / R(nx), &sn, &cs);
    const R4<R> c = coef[m];
    g.x = fma(c.x, cs, fma(-c.y, sn, g.x));
    g.y = fma(c.x, sn, fma(c.y, cs, g.y));
    g.z = fma(c.z, cs, fma(-c.w, sn, g.z));
    g.w = fma(c.z, sn, fma(c.w, cs, g.w));
  }
  return g;
}

template <typename R> __device__ __forceinline__ R4<R> r4_sum(const R4<R> &a, const R4<R> &b) {
  return R4<R>{a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w};
}

template <typename R>
__device__ inline R4<R> stir_row_entry(const R4<R> *coef, const int *kx, const int *row_start, int r, int x, int nx) {
  const R4<R> p0 = stir_entry_part<R>(coef, kx, row_start, r, x, nx, 0);
  const R4<R> p1 = stir_entry_part<R>(coef, kx, row_start, r, x, nx, 1);
  const R4<R> p2 = stir_entry_part<R>(coef, kx, row_start, r, x, nx, 2);
  const R4<R> p3 = stir_entry_part<R>(coef, kx, row_start, r, x, nx, 3);
  return r4_sum<R>(r4_sum<R>(p0, p1), r4_sum<R>(p2, p3));
}

template <typename R>
__device__ inline R4<R> stir_row_entry(const Stir<R> &s, const R4<R> *coef, int r, int x, int nx) {
  return stir_row_entry<R>(coef, s.mode_kx, s.row_start, r, x, nx);
}

// The table of step n+1 by `ncta` CTAs of a launch (this one has rank `rank`), with the
// mode coefficients, k_x and row ranges first copied to shared memory `sm` when they fit
// in `sm_bytes`.  Entry e goes to CTA e mod ncta, thread (e div ncta) mod nthr.
template <typename R>
__device__ inline void stir_table_part(const Stir<R> &s, int rank, int ncta, int tid, int nthr, int nx,
                                       unsigned char *sm, int sm_bytes) {
  if (s.nrows == 0) return;
  const R4<R> *coef = s.coef_next;
  const int *kx = s.mode_kx, *rs = s.row_start;
  const int need = s.nmodes * (int)(sizeof(R4<R>) + sizeof(int)) + (s.nrows + 1) * (int)sizeof(int);
  if (sm && need <= sm_bytes) {
    R4<R> *c2 = reinterpret_cast<R4<R> *>(sm);
    int *k2 = reinterpret_cast<int *>(c2 + s.nmodes);
    int *r2 = k2 + s.nmodes;
    for (int i = tid; i < s.nmodes; i += nthr) { c2[i] = coef[i]; k2[i] = kx[i]; }
    for (int i = tid; i <= s.nrows; i += nthr) r2[i] = rs[i];
    __syncthreads();
    coef = c2; kx = k2; rs = r2;
  }
  const long long entries = (long long)s.nrows * nx;
  for (long long e = rank + (long long)ncta * tid; e < entries; e += (long long)ncta * nthr)
    s.G_next[e] = stir_row_entry<R>(coef, kx, rs, (int)(e / nx), (int)(e % nx), nx);
}

// The per-row phase table EY_r(y) = exp(i 2 pi k_y(r) y / ny): each k_y row holds 2 eyp
// reals in blocks of 8 lattice rows; entry k (0..3) of block b holds
// (Re y, Re y+1, Im y, Im y+1) for y = 8b + 2k.  One 16-byte load then gives a thread of the
// paired step kernels (cells y and y + 1) both phases as register pairs.
__host__ __device__ __forceinline__ int ey_index(int y) { return (y >> 3) * 16 + ((y >> 1) & 3) * 4 + (y & 1); }
template <typename R> __device__ __forceinline__ R2<R> ey_at(const R *row, int y) {
  const int i = ey_index(y);
  return R2<R>{row[i], row[i + 2]};
}

// Byte sizes of the mode data a step launch copies to shared memory for the table of the
// next step: coefficients (16-byte R4 per mode for FP32, 32 for FP64), k_x and the row
// ranges, each part padded to 16 bytes (the copies are untiled bulk copies).
__host__ __device__ inline int mode_coef_bytes(int nmodes, int rbytes) { return nmodes * 4 * rbytes; }
__host__ __device__ inline int mode_kx_bytes(int nmodes) { return (nmodes * 4 + 15) / 16 * 16; }
__host__ __device__ inline int mode_rows_bytes(int nrows) { return ((nrows + 1) * 4 + 15) / 16 * 16; }

// This CTA's share of the table of step n+1 from mode data already in shared memory.
// Entry e goes to CTA e mod ncta.  Within the CTA, quads of lanes take the entries (dealt
// round-robin over the warps) and split each entry's modes four ways, summing with two
// shuffles: a row of the shell holds up to a dozen modes, and the longest entry, not the
// number of entries, sets the time.  Every thread reaches the shuffles the same number of
// times (all lanes of a warp take part).
template <typename R>
__device__ inline void stir_table_staged(const Stir<R> &s, int rank, int ncta, int tid, int nthr, int nx,
                                         const R4<R> *coef, const int *kx, const int *rs) {
  const int nwarps = nthr >> 5, nquads = nthr >> 2;
  const int lane = tid & 31, warp = tid >> 5, l4 = tid & 3;
  const int quad = warp + nwarps * (lane >> 2);  // quads of one warp are nwarps apart
  const long long entries = (long long)s.nrows * nx;
  const long long mine = entries > rank ? (entries - 1 - rank) / ncta + 1 : 0;  // this CTA's entries
  for (long long base = 0; base < mine; base += nquads) {
    const long long i = base + quad;
    R4<R> g{R(0), R(0), R(0), R(0)};
    int r = 0, x = 0;
    if (i < mine) {
      const long long e = rank + i * ncta;
      r = (int)(e / nx);
      x = (int)(e % nx);
      g = stir_entry_part<R>(coef, kx, rs, r, x, nx, l4);
    }
    // lane 0 of the quad ends with (p0 + p1) + (p2 + p3), as stir_row_entry
#pragma unroll
    for (int off = 1; off < 4; off <<= 1) {
      R4<R> o;
      o.x = __shfl_xor_sync(0xffffffffu, g.x, off);
      o.y = __shfl_xor_sync(0xffffffffu, g.y, off);
      o.z = __shfl_xor_sync(0xffffffffu, g.z, off);
      o.w = __shfl_xor_sync(0xffffffffu, g.w, off);
      g = r4_sum<R>(g, o);
    }
    if (i < mine && l4 == 0) s.G_next[(long long)r * nx + x] = g;
  }
}

// Mode m of step n in FP32 (the draws of the FP32-compute paths; the uniform u_j and
// the Box-Muller transform in single precision, about 1e-7 relative).
__device__ inline void stir_draw_f32(unsigned long long seed, long long n, int m, float amp, float out[4]) {
  uint32_t c[4] = {(uint32_t)(n & 0xffffffffll), (uint32_t)m, (uint32_t)((unsigned long long)n >> 32), 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xffffffffull), (uint32_t)(seed >> 32));
  float u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) u[j] = ((float)c[j] + 0.5f) * 2.3283064365386962890625e-10f;
  const float a = amp * sqrtf(-2.0f * logf(u[0])) * cospif(2.0f * u[1]);
  float sphi, cphi, spsi, cpsi;
  sincospif(2.0f * u[2], &sphi, &cphi);
  sincospif(2.0f * u[3], &spsi, &cpsi);
  out[0] = a * cpsi * cphi; out[1] = a * cpsi * sphi;
  out[2] = a * spsi * cphi; out[3] = a * spsi * sphi;
}

// Philox draws of step n+2: mode m by one thread of the CTA of rank m, m + ncta, ...
// (FP64 arithmetic in the FP64 path, FP32 in the others: GB300's FP64 rate is 1/64 of
// FP32, and the draws sit on the critical path of the CTAs that make them).
template <typename R>
__device__ inline void stir_draws_part(const Stir<R> &s, int rank, int ncta) {
  for (int m = rank; m < s.nmodes; m += ncta) {
    if constexpr (sizeof(R) == 8) {
      double c[4];
      stir_draw(s.seed, s.step_new, m, s.mode_scale ? s.amp * s.mode_scale[m] : s.amp, c);
      s.coef_new[m] = R4<R>{(R)c[0], (R)c[1], (R)c[2], (R)c[3]};
    } else {
      float c[4];
      stir_draw_f32(s.seed, s.step_new, m, (float)(s.mode_scale ? s.amp * s.mode_scale[m] : s.amp), c);
      s.coef_new[m] = R4<R>{c[0], c[1], c[2], c[3]};
    }
  }
}

// ---------------------------------------------------------------------------
// Arithmetic helpers: exact in FP64, hardware approximations (<= 2 ulp) in FP32.
// ---------------------------------------------------------------------------
template <typename T> struct FM;
template <> struct FM<double> {
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / sqrt(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double qroot(double x) { return sqrt(sqrt(x)); }
  static __device__ __forceinline__ double croot(double x) { return cbrt(x); }
};
template <> struct FM<float> {
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
  static __device__ __forceinline__ float qroot(float x) { return rsqrtf(rsqrtf(x)); }
  static __device__ __forceinline__ float croot(float x) { return cbrtf(x); }
};

// Two FP32 lanes (two lattice cells) in one register pair: Blackwell's packed FP32
// add/multiply/FMA (__fadd2_rn, __fmul2_rn, __ffma2_rn) do both in one instruction.
struct F2 {
  float2 v;
  __device__ __forceinline__ F2() : v(make_float2(0.0f, 0.0f)) {}
  __device__ __forceinline__ explicit F2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ explicit F2(double s) : v(make_float2((float)s, (float)s)) {}
  __device__ __forceinline__ explicit F2(int s) : v(make_float2((float)s, (float)s)) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit F2(float2 w) : v(w) {}
  __device__ __forceinline__ F2 &operator+=(F2 o) { v = __fadd2_rn(v, o.v); return *this; }
  __device__ __forceinline__ F2 &operator-=(F2 o) { v = __ffma2_rn(o.v, make_float2(-1.0f, -1.0f), v); return *this; }
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)); }
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 fmax(F2 a, F2 b) { return F2(fmaxf(a.v.x, b.v.x), fmaxf(a.v.y, b.v.y)); }
// a / b, correctly rounded per lane
template <typename T> __device__ __forceinline__ T divide(T a, T b) { return a / b; }
__device__ __forceinline__ F2 divide(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }

template <> struct FM<F2> {
  static __device__ __forceinline__ F2 rcp(F2 x) { return F2(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y)); }
  static __device__ __forceinline__ F2 rsqrt(F2 x) { return F2(rsqrtf(x.v.x), rsqrtf(x.v.y)); }
  static __device__ __forceinline__ F2 sqrt_(F2 x) { return F2(FM<float>::sqrt_(x.v.x), FM<float>::sqrt_(x.v.y)); }
  static __device__ __forceinline__ F2 qroot(F2 x) { return F2(FM<float>::qroot(x.v.x), FM<float>::qroot(x.v.y)); }
  static __device__ __forceinline__ F2 croot(F2 x) { return F2(cbrtf(x.v.x), cbrtf(x.v.y)); }
};

// ---------------------------------------------------------------------------
// Moments.  In units of eps0, with h the normalised deviations:
//   T^00 = 1 + e,  T^0a = m_a,  T^ab = delta_ab / D_p + t_ab  (a, b in {x, y})
//   e = sum w h, m = sum w h v, t = sum w h v v, and (for the force) the third
//   moments w_abc = sum w h v_a v_b v_c.  The rest-equilibrium parts are exact.
// ---------------------------------------------------------------------------
template <typename T> struct Mom { T e, mx, my, txx, txy, tyy, wxxx, wxxy, wxyy, wyyy; };

// Generic sum over classes with compile-time coefficients.
template <typename T, typename R, int VS, bool THIRD>
__device__ __forceinline__ Mom<T> moments_generic(const R h[VSet<VS>::Q]) {
  using V = VSet<VS>;
  Mom<T> M{};
#pragma unroll
  for (int q = 0; q < V::Q; ++q) {
    const double w = V::w(q), vx = V::vx(q), vy = V::vy(q);
    const T hq = (T)h[q];
    M.e += T(w) * hq;
    if (vx != 0.0) { M.mx += T(w * vx) * hq; M.txx += T(w * vx * vx) * hq; }
    if (vy != 0.0) { M.my += T(w * vy) * hq; M.tyy += T(w * vy * vy) * hq; }
    if (vx != 0.0 && vy != 0.0) M.txy += T(w * vx * vy) * hq;
    if (THIRD) {
      if (vx != 0.0) M.wxxx += T(w * vx * vx * vx) * hq;
      if (vx != 0.0 && vy != 0.0) { M.wxxy += T(w * vx * vx * vy) * hq; M.wxyy += T(w * vx * vy * vy) * hq; }
      if (vy != 0.0) M.wyyy += T(w * vy * vy * vy) * hq;
    }
  }
  return M;
}

// The 17 folded classes of the paper's set come in four sign-symmetric groups
// {(+a,+b), (-a,+b), (-a,-b), (+a,-b)} (diagonals) or {(+a,0), (0,+a), (-a,0), (0,-a)}
// (axes).  Sums and differences within a group (a butterfly) give each moment from one
// product per group instead of one per class.
template <typename T, typename R, bool THIRD>
__device__ __forceinline__ void moments_axis_group(Mom<T> &M, double w, double a, T h0, T h1, T h2, T h3) {
  // classes (+a,0), (0,+a), (-a,0), (0,-a)
  const T sx = h0 + h2, dx = h0 - h2, sy = h1 + h3, dy = h1 - h3;
  M.e += T(w) * (sx + sy);
  M.mx += T(w * a) * dx;
  M.my += T(w * a) * dy;
  M.txx += T(w * a * a) * sx;
  M.tyy += T(w * a * a) * sy;
  if (THIRD) { M.wxxx += T(w * a * a * a) * dx; M.wyyy += T(w * a * a * a) * dy; }
}
template <typename T, typename R, bool THIRD>
__device__ __forceinline__ void moments_diag_group(Mom<T> &M, double w, double a, T h0, T h1, T h2, T h3) {
  // classes (+a,+a), (-a,+a), (-a,-a), (+a,-a)
  const T s02 = h0 + h2, d02 = h0 - h2, s13 = h1 + h3, d31 = h3 - h1;
  const T P0 = s02 + s13, Pxy = s02 - s13, Px = d02 + d31, Py = d02 - d31;
  M.e += T(w) * P0;
  M.txx += T(w * a * a) * P0;
  M.tyy += T(w * a * a) * P0;
  M.mx += T(w * a) * Px;
  M.my += T(w * a) * Py;
  M.txy += T(w * a * a) * Pxy;
  if (THIRD) {
    M.wxxx += T(w * a * a * a) * Px;
    M.wxyy += T(w * a * a * a) * Px;
    M.wxxy += T(w * a * a * a) * Py;
    M.wyyy += T(w * a * a * a) * Py;
  }
}

template <typename T, typename R, int VS, bool THIRD>
__device__ __forceinline__ Mom<T> moments_of(const R h[VSet<VS>::Q]) {
  if constexpr (VS == 3) {
    using V = VSet<3>;
    Mom<T> M{};
    M.e = T(V::w(0)) * (T)h[0];
    moments_axis_group<T, R, THIRD>(M, V::w(1), 1.0, (T)h[1], (T)h[2], (T)h[3], (T)h[4]);
    moments_diag_group<T, R, THIRD>(M, V::w(5), RLBM_S2, (T)h[5], (T)h[6], (T)h[7], (T)h[8]);
    moments_axis_group<T, R, THIRD>(M, V::w(9), RLBM_S2, (T)h[9], (T)h[10], (T)h[11], (T)h[12]);
    moments_diag_group<T, R, THIRD>(M, V::w(13), RLBM_S3, (T)h[13], (T)h[14], (T)h[15], (T)h[16]);
    return M;
  } else {
    return moments_generic<T, R, VS, THIRD>(h);
  }
}

// ---------------------------------------------------------------------------
// Landau matching: the timelike eigenvector u = gamma (1, v) of T^mu_nu on the
// (t, x, y) block solves  R(v) = m - T^{ab} v_b - (T^00 - m.v) v = 0.  Starting point:
// the exact solution for an ideal fluid with the same T^00 and T^0a (for D_p = 3,
// |m| / T^00 = 4 v / (3 + v^2); for D_p = 2, 3 v / (2 + v^2)), then Newton steps.
// Returns false when the last Newton step is not small (|dv| > tol (|v| + 1e-6)) or
// the result is not a subluminal flow with positive energy density.
// ---------------------------------------------------------------------------
template <typename T, int VS>
__device__ __forceinline__ bool landau(const Mom<T> &M, int maxit, T tol, T &vx, T &vy) {
  constexpr T dinv = T(1.0 / VSet<VS>::DP);
  const T T00 = T(1) + M.e;
  const T i00 = FM<T>::rcp(T00);
  const T ax = M.mx * i00, ay = M.my * i00, m2 = ax * ax + ay * ay;
  T c;
  if (VS == 3) c = T(3) * FM<T>::rcp(T(2) + FM<T>::sqrt_(fmax(T(4) - T(3) * m2, T(0))));
  else c = T(4) * FM<T>::rcp(T(3) + FM<T>::sqrt_(fmax(T(9) - T(8) * m2, T(0))));
  vx = c * ax;
  vy = c * ay;
  const T Txx = dinv + M.txx, Txy = M.txy, Tyy = dinv + M.tyy;
  T d2 = T(0);
  for (int it = 0; it < maxit; ++it) {
    const T E = T00 - (M.mx * vx + M.my * vy);
    const T rx = M.mx - (Txx * vx + Txy * vy) - E * vx;
    const T ry = M.my - (Txy * vx + Tyy * vy) - E * vy;
    // J = dR/dv = -T^{ab} + v_a m_b - E delta_ab
    const T jxx = -Txx + vx * M.mx - E, jxy = -Txy + vx * M.my;
    const T jyx = -Txy + vy * M.mx, jyy = -Tyy + vy * M.my - E;
    const T idet = FM<T>::rcp(jxx * jyy - jxy * jyx);
    const T dx = (jxy * ry - jyy * rx) * idet;
    const T dy = (jyx * rx - jxx * ry) * idet;
    vx += dx;
    vy += dy;
    d2 = dx * dx + dy * dy;
    if constexpr (sizeof(T) == 8) {
      if (d2 <= 1e-32 * (vx * vx + vy * vy) + 1e-300) break;
    } else {
      if (d2 <= tol * tol * (T(1e-6) + vx * vx + vy * vy)) break;
    }
  }
  const T v2 = vx * vx + vy * vy;
  const T lim = tol * (T(1e-6) + v2);
  return (v2 < T(1)) && (T00 - (M.mx * vx + M.my * vy) > T(0)) && (d2 <= tol * lim);
}

// Macroscopic result of one cell (eps^ = eps / eps0, u^mu = gamma (1, v)).
template <typename T> struct Macro { T eps_m1, u0, ux, uy, vx, vy; bool ok; };

template <typename T, int VS>
__device__ __forceinline__ Macro<T> macro_from(const Mom<T> &M, int maxit, T tol) {
  Macro<T> r;
  T vx, vy;
  const bool ok = landau<T, VS>(M, maxit, tol, vx, vy);
  const T v2 = vx * vx + vy * vy;
  const T gam = FM<T>::rsqrt(T(1) - v2);
  r.eps_m1 = M.e - (M.mx * vx + M.my * vy);
  r.u0 = gam; r.ux = gam * vx; r.uy = gam * vy; r.vx = vx; r.vy = vy;
  r.ok = ok && (T(1) + r.eps_m1 > T(0)) && isfinite(r.eps_m1) && isfinite(gam);
  return r;
}

// Landau matching of one cell in the compute type; the FP32 path re-solves in FP64
// (moments re-summed in FP64 from the same h) when its two Newton steps have not
// converged or |v|^2 exceeds vmax2.
template <typename R, int VS>
__device__ __forceinline__ Macro<R> cell_macro(const R h[VSet<VS>::Q], const Mom<R> &M, R vmax2) {
  if constexpr (sizeof(R) == 8) {
    return macro_from<double, VS>(M, 40, 1e-12);
  } else {
    Macro<float> m = macro_from<float, VS>(M, 4, 3e-4f);
    if (!m.ok || m.vx * m.vx + m.vy * m.vy > vmax2) {
      const Mom<double> Md = moments_of<double, R, VS, false>(h);
      const Macro<double> d = macro_from<double, VS>(Md, 40, 1e-12);
      m.eps_m1 = (float)d.eps_m1; m.u0 = (float)d.u0; m.ux = (float)d.ux; m.uy = (float)d.uy;
      m.vx = (float)d.vx; m.vy = (float)d.vy; m.ok = d.ok;
    }
    return m;
  }
}

// Landau matching of two cells at once: the Newton steps of `landau` on both lanes, each
// lane keeping its value from the step at which it converged (so a cell's result does not
// depend on the cell it is paired with); a lane that has not converged, or whose |v|^2
// exceeds vmax2, is re-solved in FP64 from the same populations.
template <int VS>
__device__ __forceinline__ Macro<F2> cell_macro_pair(const F2 h[VSet<VS>::Q], const Mom<F2> &M, float vmax2) {
  constexpr float dinv = 1.0f / VSet<VS>::DP;
  const float tol = 3e-4f;
  const F2 one(1.0f);
  const F2 T00 = one + M.e;
  const F2 i00 = FM<F2>::rcp(T00);
  const F2 ax = M.mx * i00, ay = M.my * i00, m2 = fma(ax, ax, ay * ay);
  F2 c;
  if (VS == 3) c = F2(3.0f) * FM<F2>::rcp(F2(2.0f) + FM<F2>::sqrt_(fmax(fma(F2(-3.0f), m2, F2(4.0f)), F2(0.0f))));
  else c = F2(4.0f) * FM<F2>::rcp(F2(3.0f) + FM<F2>::sqrt_(fmax(fma(F2(-8.0f), m2, F2(9.0f)), F2(0.0f))));
  F2 vx = c * ax, vy = c * ay;
  const F2 Txx = F2(dinv) + M.txx, Txy = M.txy, Tyy = F2(dinv) + M.tyy;
  bool convA = false, convB = false;
  for (int it = 0; it < 4; ++it) {
    const F2 E = T00 - fma(M.mx, vx, M.my * vy);
    const F2 rx = M.mx - fma(Txx, vx, Txy * vy) - E * vx;
    const F2 ry = M.my - fma(Txy, vx, Tyy * vy) - E * vy;
    const F2 jxx = fma(vx, M.mx, -Txx) - E, jxy = fma(vx, M.my, -Txy);
    const F2 jyx = fma(vy, M.mx, -Txy), jyy = fma(vy, M.my, -Tyy) - E;
    const F2 idet = FM<F2>::rcp(jxx * jyy - jxy * jyx);
    const F2 dx = (jxy * ry - jyy * rx) * idet;
    const F2 dy = (jyx * rx - jxx * ry) * idet;
    vx += F2(convA ? 0.0f : dx.v.x, convB ? 0.0f : dx.v.y);
    vy += F2(convA ? 0.0f : dy.v.x, convB ? 0.0f : dy.v.y);
    const F2 d2 = fma(dx, dx, dy * dy), lim = F2(tol * tol) * (F2(1e-6f) + fma(vx, vx, vy * vy));
    convA = convA || d2.v.x <= lim.v.x;
    convB = convB || d2.v.y <= lim.v.y;
    if (convA && convB) break;
  }
  const F2 v2 = fma(vx, vx, vy * vy);
  const F2 E = T00 - fma(M.mx, vx, M.my * vy);
  const bool okA = convA && v2.v.x < vmax2 && E.v.x > 0.0f, okB = convB && v2.v.y < vmax2 && E.v.y > 0.0f;
  Macro<F2> r;
  const F2 gam = FM<F2>::rsqrt(one - v2);
  r.eps_m1 = M.e - fma(M.mx, vx, M.my * vy);
  r.u0 = gam; r.ux = gam * vx; r.uy = gam * vy; r.vx = vx; r.vy = vy;
  r.ok = true;
  if (!okA || !okB) {
    for (int lane = 0; lane < 2; ++lane) {
      if (lane == 0 ? okA : okB) continue;
      float hl[VSet<VS>::Q];
#pragma unroll
      for (int q = 0; q < VSet<VS>::Q; ++q) hl[q] = lane == 0 ? h[q].v.x : h[q].v.y;
      const Mom<double> Md = moments_of<double, float, VS, false>(hl);
      const Macro<double> d = macro_from<double, VS>(Md, 40, 1e-12);
      float *dst[6] = {lane ? &r.eps_m1.v.y : &r.eps_m1.v.x, lane ? &r.u0.v.y : &r.u0.v.x,
                       lane ? &r.ux.v.y : &r.ux.v.x, lane ? &r.uy.v.y : &r.uy.v.x,
                       lane ? &r.vx.v.y : &r.vx.v.x, lane ? &r.vy.v.y : &r.vy.v.x};
      *dst[0] = (float)d.eps_m1; *dst[1] = (float)d.u0; *dst[2] = (float)d.ux;
      *dst[3] = (float)d.uy; *dst[4] = (float)d.vx; *dst[5] = (float)d.vy;
      r.ok = r.ok && d.ok;
    }
  }
  r.ok = r.ok && isfinite(r.eps_m1.v.x) && isfinite(r.eps_m1.v.y) && (1.0f + r.eps_m1.v.x > 0.0f) &&
         (1.0f + r.eps_m1.v.y > 0.0f);
  return r;
}

// ---------------------------------------------------------------------------
// Collision and force of one cell, as per-class polynomials in v_i:
//   h*_i = h_i + omega (u^0 - u.v_i)(h_eq,i - h_i) + dt S_i / (w_i eps0)
//   h_eq,i = (eps^ - 1) + CA eps^ u^0 (u.v_i) + CB eps^ (u.v_i)^2 - CC eps^ |u|^2
// (the equilibrium of Eq. rel_pdf_exp_coef with T_eq = (eps + P) u u - P g), so with
// t = u.v_i:  h*_i = h_i (1 - omega u^0 + omega t) + p0 + p1 t + p2 t^2 + p3 t^3 + S_i.
// The force (Eq. forceTerm with App. B's coefficients, prefactor -6/T0 dt):
//   S_i = fpref [ F.M1 / 4 - (M0 / 2) F.v_i + 5/4 v_i.B.v_i - 5/2 (F.v_i)(v_i.M1) ]
//       = s0 + s1.v_i + v_i.S2.v_i + szz v_z,i^2
// with B_ab = sum f (F.v) v_a v_b and B_zz = F.M1 - B_xx - B_yy (|v| = 1).
// ---------------------------------------------------------------------------
template <typename R> struct Coll {
  R ux, uy, k0, om, p0, p1, p2, p3;
  R s0, s1x, s1y, sxx, sxy2, syy, szz;
};

// one: the scale of the collision's output (the stored form's HScale::up, with omega0 and
// fpref passed already multiplied by it; every coefficient below is then scaled by it too).
template <typename R, int VS, bool FORCE>
__device__ __forceinline__ Coll<R> coll_coeffs(const Mom<R> &M, const Macro<R> &m, R omega0, R fpref, R Fx, R Fy,
                                               R one = R(1)) {
  using V = VSet<VS>;
  Coll<R> c;
  const R epsh = R(1) + m.eps_m1;
  const R om = VS == 3 ? omega0 * FM<R>::qroot(epsh) : omega0 * FM<R>::croot(epsh);
  const R u2 = m.ux * m.ux + m.uy * m.uy;
  const R ca = R(V::CA) * epsh * m.u0, cb = R(V::CB) * epsh, cc = m.eps_m1 - R(V::CC) * epsh * u2;
  c.ux = m.ux; c.uy = m.uy; c.om = om;
  c.k0 = one - om * m.u0;
  c.p0 = om * m.u0 * cc;
  c.p1 = om * (m.u0 * ca - cc);
  c.p2 = om * (m.u0 * cb - ca);
  c.p3 = -om * cb;
  c.s0 = c.s1x = c.s1y = c.sxx = c.sxy2 = c.syy = c.szz = R(0);
  if (FORCE) {
    const R FM1 = Fx * M.mx + Fy * M.my, M0 = R(1) + M.e;
    const R Bxx = Fx * M.wxxx + Fy * M.wxxy;
    const R Bxy = Fx * M.wxxy + Fy * M.wxyy;
    const R Byy = Fx * M.wxyy + Fy * M.wyyy;
    const R Bzz = FM1 - Bxx - Byy;
    const R f54 = R(1.25) * fpref;
    c.s0 = R(0.25) * fpref * FM1;
    c.s1x = R(-0.5) * fpref * M0 * Fx;
    c.s1y = R(-0.5) * fpref * M0 * Fy;
    c.sxx = f54 * (Bxx - R(2) * Fx * M.mx);
    c.sxy2 = R(2) * f54 * (Bxy - Fx * M.my - Fy * M.mx);
    c.syy = f54 * (Byy - R(2) * Fy * M.my);
    c.szz = f54 * Bzz;
  }
  c.s0 += c.p0;
  return c;
}

template <typename R, int VS, bool FORCE>
__device__ __forceinline__ R collide_class(const Coll<R> &c, int q, R h) {
  using V = VSet<VS>;
  const double vx = V::vx(q), vy = V::vy(q), vz2 = V::vz2(q);
  R t = R(0);
  if (vx != 0.0) t = c.ux * R(vx);
  if (vy != 0.0) t = fma(c.uy, R(vy), t);
  R acc = c.s0;
  if (FORCE) {
    if (vx != 0.0) acc = fma(c.s1x, R(vx), acc);
    if (vy != 0.0) acc = fma(c.s1y, R(vy), acc);
    if (vx != 0.0) acc = fma(c.sxx, R(vx * vx), acc);
    if (vx != 0.0 && vy != 0.0) acc = fma(c.sxy2, R(vx * vy), acc);
    if (vy != 0.0) acc = fma(c.syy, R(vy * vy), acc);
    if (vz2 != 0.0) acc = fma(c.szz, R(vz2), acc);
  }
  if (vx != 0.0 || vy != 0.0) acc = fma(t, fma(t, fma(t, c.p3, c.p2), c.p1), acc);
  const R k = (vx != 0.0 || vy != 0.0) ? fma(c.om, t, c.k0) : c.k0;
  return fma(h, k, acc);
}

// All classes of a cell.  For the paper's set the classes of a sign group
// {(+a,+b), (-a,+b), (-a,-b), (+a,-b)} share a u-projection pair (a u^x, b u^y) and the
// even part of the force polynomial; only signs differ between the four members.
template <typename R, bool FORCE>
__device__ __forceinline__ void collide_group(const Coll<R> &c, double a, double b, double vz2, R h0, R h1, R h2,
                                              R h3, R &o0, R &o1, R &o2, R &o3) {
  const R A = c.ux * R(a), B = c.uy * R(b);
  R even = c.s0, X = R(0), Y = R(0), XY = R(0);
  if (FORCE) {
    even = fma(c.sxx, R(a * a), even);
    if (b != 0.0) even = fma(c.syy, R(b * b), even);
    if (vz2 != 0.0) even = fma(c.szz, R(vz2), even);
    X = c.s1x * R(a);
    if (b != 0.0) { Y = c.s1y * R(b); XY = c.sxy2 * R(a * b); }
  }
  auto one = [&](R t, R force, R hq) {
    const R acc = fma(t, fma(t, fma(t, c.p3, c.p2), c.p1), force);
    return fma(hq, fma(c.om, t, c.k0), acc);
  };
  if (b != 0.0) {  // diagonal group: (+a,+b), (-a,+b), (-a,-b), (+a,-b)
    const R e0 = even + XY, e1 = even - XY;
    o0 = one(A + B, e0 + (X + Y), h0);
    o1 = one(B - A, e1 + (Y - X), h1);
    o2 = one(-(A + B), e0 - (X + Y), h2);
    o3 = one(A - B, e1 + (X - Y), h3);
  } else {  // axis group: (+a,0), (0,+a), (-a,0), (0,-a)
    R evx = even, evy = c.s0;
    R Yv = R(0);
    if (FORCE) {
      evy = fma(c.syy, R(a * a), c.s0);
      if (vz2 != 0.0) evy = fma(c.szz, R(vz2), evy);
      Yv = c.s1y * R(a);
    }
    const R By = c.uy * R(a);
    o0 = one(A, evx + X, h0);
    o1 = one(By, evy + Yv, h1);
    o2 = one(-A, evx - X, h2);
    o3 = one(-By, evy - Yv, h3);
  }
}

template <typename R, int VS, bool FORCE>
__device__ __forceinline__ void collide_all(const Coll<R> &c, const R h[VSet<VS>::Q], R hn[VSet<VS>::Q]) {
  if constexpr (VS == 3) {
    // class 0: v = (0, 0), v_z^2 = 1
    hn[0] = fma(h[0], c.k0, FORCE ? fma(c.szz, R(1), c.s0) : c.s0);
    collide_group<R, FORCE>(c, 1.0, 0.0, 0.0, h[1], h[2], h[3], h[4], hn[1], hn[2], hn[3], hn[4]);
    collide_group<R, FORCE>(c, RLBM_S2, RLBM_S2, 0.0, h[5], h[6], h[7], h[8], hn[5], hn[6], hn[7], hn[8]);
    collide_group<R, FORCE>(c, RLBM_S2, 0.0, 0.5, h[9], h[10], h[11], h[12], hn[9], hn[10], hn[11], hn[12]);
    collide_group<R, FORCE>(c, RLBM_S3, RLBM_S3, 1.0 / 3.0, h[13], h[14], h[15], h[16], hn[13], hn[14], hn[15], hn[16]);
  } else {
#pragma unroll
    for (int q = 0; q < VSet<VS>::Q; ++q) hn[q] = collide_class<R, VS, FORCE>(c, q, h[q]);
  }
}

}  // namespace rlbm
