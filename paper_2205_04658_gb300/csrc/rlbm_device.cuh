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

enum : unsigned { ERR_UNSTABLE = 1u, ERR_UNPHYSICAL = 2u };

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
template <typename S, typename R> __device__ __forceinline__ R load_h(const S *p) { return (R)__ldg(p); }
template <> __device__ __forceinline__ float load_h<__half, float>(const __half *p) {
  return __half2float(__ldg(p));
}
template <> __device__ __forceinline__ float load_h<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
  return __bfloat162float(__ldg(p));
}
template <typename S, typename R> __device__ __forceinline__ S store_h(R v) { return (S)v; }
template <> __device__ __forceinline__ __half store_h<__half, float>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 store_h<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

template <typename S> struct RealOf { using type = float; };
template <> struct RealOf<double> { using type = double; };

// ---------------------------------------------------------------------------
// Parameters
// ---------------------------------------------------------------------------
template <typename R> struct alignas(16) R4 { R x, y, z, w; };
template <typename R> struct alignas(2 * sizeof(R)) R2 { R x, y; };

template <typename R> struct Geometry {
  int nx, ny, pitch;
  long long plane;          // elements per plane (pitch * ny)
  const uint16_t *nbmask;   // bit 4: cell solid; bit (dy+1)*3+(dx+1): neighbour (x+dx, y+dy) solid
  R beta[17][4];            // bilinear weights of corners (0,0), (s_x,0), (0,s_y), (s_x,s_y)
};

template <typename R> struct Physics {
  R omega0;        // dt T0 / (TAU_NUM eta/s): relaxation factor at eps = eps0
  R fpref;         // -6 dt / T0: force prefactor including dt
  R body_x, body_y;
  double vmax2;    // FP32 path: |v|^2 above which Landau runs in FP64
  int has_force;   // any force (body or stirring)
};

template <typename R> struct Stir {
  int nrows;               // distinct k_y of the shell (0 = no stirring)
  int nmodes;
  const R4<R> *G_cur;      // [nrows][nx]: (Gx.re, Gx.im, Gy.re, Gy.im) of this step
  const R2<R> *EY;         // [nrows][ny]: exp(i 2 pi k_y(row) y / ny)
  // pipelined preparation of the next steps (done by the same launch)
  R4<R> *G_next;           // [nrows][nx] of step n+1
  const R4<R> *coef_next;  // [nmodes]: (cx.re, cx.im, cy.re, cy.im) of step n+1
  R4<R> *coef_new;         // [nmodes] of step n+2 (written)
  const int *mode_kx;      // [nmodes]
  const int *mode_ky;      // [nmodes]
  const int *row_start;    // [nrows+1] mode range of each row (modes sorted by k_y)
  const R2<R> *EX;         // [nx]: exp(i 2 pi j / nx)
  unsigned long long seed;
  long long step_new;      // n + 2
  double amp;
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

// One entry of the per-row stirring table of a step:
//   G_r(x) = sum_{m in row r} (cx_m, cy_m) exp(i 2 pi k_x,m x / nx).
template <typename R>
__device__ inline R4<R> stir_row_entry(const Stir<R> &s, const R4<R> *coef, int r, int x, int nx) {
  R4<R> g{R(0), R(0), R(0), R(0)};
  for (int m = s.row_start[r]; m < s.row_start[r + 1]; ++m) {
    long long j = ((long long)s.mode_kx[m] * x) % nx;
    if (j < 0) j += nx;
    const R2<R> e = s.EX[j];
    const R4<R> c = coef[m];
    g.x += c.x * e.x - c.y * e.y;
    g.y += c.x * e.y + c.y * e.x;
    g.z += c.z * e.x - c.w * e.y;
    g.w += c.z * e.y + c.w * e.x;
  }
  return g;
}

// Work a step launch does for the following steps: thread t < nrows*nx builds one
// entry of G for step n+1, thread t < nmodes draws mode t of step n+2.
template <typename R>
__device__ inline void stir_prepare(const Stir<R> &s, long long t, int nx) {
  if (s.nrows == 0) return;
  if (t < (long long)s.nrows * nx) {
    const int r = (int)(t / nx), x = (int)(t % nx);
    s.G_next[t] = stir_row_entry<R>(s, s.coef_next, r, x, nx);
  }
  if (t < s.nmodes) {
    double c[4];
    stir_draw(s.seed, s.step_new, (int)t, s.amp, c);
    s.coef_new[t] = R4<R>{(R)c[0], (R)c[1], (R)c[2], (R)c[3]};
  }
}

// ---------------------------------------------------------------------------
// Streaming: bilinear pull of every class with bounce-back (solid source corners
// contribute the reversed population of the receiving cell).
// ---------------------------------------------------------------------------
template <typename S, typename R, int VS, bool MASK>
__device__ __forceinline__ void pull(const S *__restrict__ fin, const Geometry<R> &g, int x, int y,
                                     unsigned nb, R h[VSet<VS>::Q]) {
  constexpr int Q = VSet<VS>::Q;
  const int xm = x == 0 ? g.nx - 1 : x - 1;
  const int xp = x == g.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? g.ny - 1 : y - 1;
  const int yp = y == g.ny - 1 ? 0 : y + 1;
  R c[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) c[q] = load_h<S, R>(fin + q * g.plane + (long long)y * g.pitch + x);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int sx = sgnx<VS>(q), sy = sgny<VS>(q);
    const S *pl = fin + q * g.plane;
    const int cx = sx > 0 ? xm : xp;        // source column x - s_x
    const int ry = sy > 0 ? ym : yp;        // source row    y - s_y
    R acc = g.beta[q][0] * c[q];
    if (sx != 0) {
      const bool solid = MASK && ((nb >> (4 - sx)) & 1u);
      const R v = solid ? c[VSet<VS>::opp(q)] : load_h<S, R>(pl + (long long)y * g.pitch + cx);
      acc += g.beta[q][1] * v;
    }
    if (sy != 0) {
      const bool solid = MASK && ((nb >> (4 - 3 * sy)) & 1u);
      const R v = solid ? c[VSet<VS>::opp(q)] : load_h<S, R>(pl + (long long)ry * g.pitch + x);
      acc += g.beta[q][2] * v;
    }
    if (sx != 0 && sy != 0) {
      const bool solid = MASK && ((nb >> (4 - 3 * sy - sx)) & 1u);
      const R v = solid ? c[VSet<VS>::opp(q)] : load_h<S, R>(pl + (long long)ry * g.pitch + cx);
      acc += g.beta[q][3] * v;
    }
    h[q] = acc;
  }
}

// ---------------------------------------------------------------------------
// Moments and Landau matching.  In units of eps0:
//   T^00 = 1 + e,  T^0a = m_a,  T^ab = delta_ab / 3 + t_ab  (a, b in {x, y})
// with e = sum w h, m = sum w h v, t = sum w h v v (the rest-equilibrium parts are
// exact constants).  Landau: the timelike eigenvector u = gamma (1, v) of T^mu_nu on
// the (t, x, y) block solves  R(v) = m - T^{ab} v_b - (T^00 - m.v) v = 0  (2-D Newton).
// ---------------------------------------------------------------------------
template <typename T> struct Mom { T e, mx, my, txx, txy, tyy; };

template <typename T, typename R, int VS>
__device__ __forceinline__ Mom<T> moments_of(const R h[VSet<VS>::Q]) {
  constexpr int Q = VSet<VS>::Q;
  Mom<T> M{T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const T wh = T(VSet<VS>::w(q)) * (T)h[q];
    const T vx = T(VSet<VS>::vx(q)), vy = T(VSet<VS>::vy(q));
    M.e += wh;
    if (vx != T(0)) M.mx += wh * vx;
    if (vy != T(0)) M.my += wh * vy;
    if (vx != T(0)) M.txx += wh * (vx * vx);
    if (vx != T(0) && vy != T(0)) M.txy += wh * (vx * vy);
    if (vy != T(0)) M.tyy += wh * (vy * vy);
  }
  return M;
}

// Returns false when Newton did not converge to |R| <= tol * T^00 (or |v| >= 1).
template <typename T, int VS>
__device__ __forceinline__ bool landau(const Mom<T> &M, int maxit, T tol, T &vx, T &vy) {
  constexpr T third = T(1.0 / VSet<VS>::DP);
  const T T00 = T(1) + M.e;
  const T Txx = third + M.txx, Txy = M.txy, Tyy = third + M.tyy;
  const T s = T(VSet<VS>::DP) / T(VSet<VS>::DP + 1) / T00;  // small-v start: v = D m / ((D+1) T^00)
  vx = s * M.mx;
  vy = s * M.my;
  T rx = T(0), ry = T(0);
  for (int it = 0; it < maxit; ++it) {
    const T E = T00 - (M.mx * vx + M.my * vy);
    rx = M.mx - (Txx * vx + Txy * vy) - E * vx;
    ry = M.my - (Txy * vx + Tyy * vy) - E * vy;
    // J = dR/dv = -T^{ab} + v_a m_b - E delta_ab
    const T jxx = -Txx + vx * M.mx - E, jxy = -Txy + vx * M.my;
    const T jyx = -Txy + vy * M.mx, jyy = -Tyy + vy * M.my - E;
    const T det = jxx * jyy - jxy * jyx;
    const T dx = -(jyy * rx - jxy * ry) / det;
    const T dy = -(-jyx * rx + jxx * ry) / det;
    vx += dx;
    vy += dy;
    if (dx * dx + dy * dy <= tol * tol * (T(1e-30) + vx * vx + vy * vy)) { rx = ry = T(0); break; }
  }
  const T E = T00 - (M.mx * vx + M.my * vy);
  rx = M.mx - (Txx * vx + Txy * vy) - E * vx;
  ry = M.my - (Txy * vx + Tyy * vy) - E * vy;
  const T v2 = vx * vx + vy * vy;
  return (v2 < T(1)) && (E > T(0)) && (sqrt(rx * rx + ry * ry) <= T(64) * tol * T00);
}

// Macroscopic result of one cell (eps^ = eps / eps0, u^mu = gamma (1, v)).
template <typename T> struct Macro { T eps_m1, u0, ux, uy, vx, vy; bool ok; };

template <typename T, int VS>
__device__ __forceinline__ Macro<T> macro_from(const Mom<T> &M, int maxit, T tol) {
  Macro<T> r;
  T vx, vy;
  const bool ok = landau<T, VS>(M, maxit, tol, vx, vy);
  const T v2 = vx * vx + vy * vy;
  const T gam = T(1) / sqrt(T(1) - v2);
  r.eps_m1 = M.e - (M.mx * vx + M.my * vy);
  r.u0 = gam; r.ux = gam * vx; r.uy = gam * vy; r.vx = vx; r.vy = vy;
  r.ok = ok && (T(1) + r.eps_m1 > T(0)) && isfinite(r.eps_m1) && isfinite(gam);
  return r;
}

// Landau matching of one cell in the storage's compute type; the FP32 path re-solves
// in FP64 (moments re-summed in FP64 from the same h) when its Newton solve fails or
// |v|^2 exceeds vmax2.
template <typename R, int VS>
__device__ __forceinline__ Macro<R> cell_macro(const R h[VSet<VS>::Q], const Mom<R> &M, double vmax2) {
  if constexpr (sizeof(R) == 8) {
    return macro_from<double, VS>(M, 40, 1e-15);
  } else {
    Macro<float> m = macro_from<float, VS>(M, 8, 2e-7f);
    if (!m.ok || (double)(m.vx * m.vx + m.vy * m.vy) > vmax2) {
      const Mom<double> Md = moments_of<double, R, VS>(h);
      const Macro<double> d = macro_from<double, VS>(Md, 40, 1e-15);
      m.eps_m1 = (float)d.eps_m1; m.u0 = (float)d.u0; m.ux = (float)d.ux; m.uy = (float)d.uy;
      m.vx = (float)d.vx; m.vy = (float)d.vy; m.ok = d.ok;
    }
    return m;
  }
}

}  // namespace rlbm
