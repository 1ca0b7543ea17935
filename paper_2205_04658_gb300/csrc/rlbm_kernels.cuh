// Kernels of the relativistic lattice Boltzmann update (arXiv 2205.04658) and the
// host launchers of one storage type.  Included once per storage type by
// rlbm_kernels_<type>.cu, which defines RLBM_STORE and RLBM_SUFFIX.
#pragma once

#include "rlbm_device.cuh"
#include "rlbm_launch.h"

namespace rlbm {

// ---------------------------------------------------------------------------
// The fused step (procedure items 2-5 of Sec. "The Standard/Classical LBM", with
// the driving term of Sec. "The Driving Term"): pull-stream f*_n -> f_n, moments,
// Landau matching, equilibrium, Anderson-Witting relaxation, projected force, store
// f*_{n+1}.  One thread per cell.
// ---------------------------------------------------------------------------
template <typename S, int VS, bool MASK>
__global__ void __launch_bounds__(256)
step_kernel(const S *__restrict__ fin, S *__restrict__ fout, const Geometry<typename RealOf<S>::type> g,
            const Physics<typename RealOf<S>::type> p, const Stir<typename RealOf<S>::type> st,
            unsigned *__restrict__ err) {
  using R = typename RealOf<S>::type;
  using V = VSet<VS>;
  constexpr int Q = V::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const long long t = ((long long)(blockIdx.y * gridDim.x + blockIdx.x) * blockDim.y + threadIdx.y) * blockDim.x
                      + threadIdx.x;
  stir_prepare<R>(st, t, g.nx);
  if (x >= g.nx || y >= g.ny) return;
  unsigned nb = 0;
  if (MASK) {
    nb = g.nbmask[(long long)y * g.nx + x];
    if (nb & 16u) return;  // solid cell: holds no fluid, never read by its neighbours
  }
  R h[Q];
  pull<S, R, VS, MASK>(fin, g, x, y, nb, h);
  const Mom<R> M = moments_of<R, R, VS>(h);
  const Macro<R> m = cell_macro<R, VS>(h, M, p.vmax2);
  if (!m.ok) atomicOr(err, (R(1) + m.eps_m1 > R(0) && isfinite(m.eps_m1)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
  const R epsh = R(1) + m.eps_m1;
  const R omega = VS == 3 ? p.omega0 * sqrt(sqrt(epsh)) : p.omega0 * cbrt(epsh);
  const R u2 = m.ux * m.ux + m.uy * m.uy;
  const R ca = R(V::CA) * epsh * m.u0, cb = R(V::CB) * epsh, cc = m.eps_m1 - R(V::CC) * epsh * u2;

  // Force at this cell: uniform body force plus the stirring field
  // F(x, y) = sum_rows Re[G_r(x) exp(i 2 pi k_y,r y / ny)].
  R Fx = p.body_x, Fy = p.body_y;
  for (int r = 0; r < st.nrows; ++r) {
    const R4<R> G = st.G_cur[(long long)r * g.nx + x];
    const R2<R> E = st.EY[(long long)r * g.ny + y];
    Fx += G.x * E.x - G.y * E.y;
    Fy += G.z * E.x - G.w * E.y;
  }
  // Force moments (App. B): M0 = T^00, M1 = T^0a, B_ab = sum f (F.v) v_a v_b, B_zz from
  // the trace B_xx + B_yy + B_zz = F.M1 (|v| = 1).
  R FM1 = R(0), M0 = R(0), Bxx = R(0), Bxy = R(0), Byy = R(0), Bzz = R(0);
  if (VS == 3 && p.has_force) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const R vx = R(V::vx(q)), vy = R(V::vy(q));
      if (vx == R(0) && vy == R(0)) continue;
      const R whf = R(V::w(q)) * h[q] * (Fx * vx + Fy * vy);
      Bxx += whf * (vx * vx);
      Bxy += whf * (vx * vy);
      Byy += whf * (vy * vy);
    }
    FM1 = Fx * M.mx + Fy * M.my;
    M0 = R(1) + M.e;
    Bzz = FM1 - Bxx - Byy;
  }
  const long long o = (long long)y * g.pitch + x;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const R vx = R(V::vx(q)), vy = R(V::vy(q));
    const R uv = m.ux * vx + m.uy * vy;
    const R heq = cc + uv * (ca + cb * uv);
    R hn = h[q] + omega * (m.u0 - uv) * (heq - h[q]);
    if (VS == 3 && p.has_force) {
      const R Fv = Fx * vx + Fy * vy;
      const R vBv = vx * vx * Bxx + R(2) * vx * vy * Bxy + vy * vy * Byy + R(V::vz2(q)) * Bzz;
      const R vM1 = vx * M.mx + vy * M.my;
      hn += p.fpref * (R(0.25) * FM1 - R(0.5) * Fv * M0 + R(1.25) * vBv - R(2.5) * Fv * vM1);
    }
    fout[q * g.plane + o] = store_h<S, R>(hn);
  }
}

// ---------------------------------------------------------------------------
// Moments of the current state f_n = stream(f*_n) (procedure item 3): eps, u^x, u^y
// per cell and per-block FP64 partial sums of T^00, T^0x, T^0y, 1/2 |v|^2.  Landau
// runs in FP64 here for every storage type.
// ---------------------------------------------------------------------------
template <typename S, int VS, bool MASK>
__global__ void __launch_bounds__(256)
moments_kernel(const S *__restrict__ fin, const Geometry<typename RealOf<S>::type> g, double eps0,
               double *__restrict__ eps, double *__restrict__ ux, double *__restrict__ uy,
               double *__restrict__ partials, unsigned *__restrict__ err) {
  using R = typename RealOf<S>::type;
  constexpr int Q = VSet<VS>::Q;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (x < g.nx && y < g.ny) {
    const long long c = (long long)y * g.nx + x;
    unsigned nb = MASK ? g.nbmask[c] : 0u;
    if (MASK && (nb & 16u)) {
      eps[c] = 0.0; ux[c] = 0.0; uy[c] = 0.0;
    } else {
      R h[Q];
      pull<S, R, VS, MASK>(fin, g, x, y, nb, h);
      const Mom<double> M = moments_of<double, R, VS>(h);
      const Macro<double> m = macro_from<double, VS>(M, 40, 1e-15);
      if (!m.ok) atomicOr(err, (1.0 + m.eps_m1 > 0.0 && isfinite(m.eps_m1)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
      eps[c] = eps0 * (1.0 + m.eps_m1);
      ux[c] = m.ux;
      uy[c] = m.uy;
      acc[0] = eps0 * (1.0 + M.e);
      acc[1] = eps0 * M.mx;
      acc[2] = eps0 * M.my;
      acc[3] = 0.5 * (m.vx * m.vx + m.vy * m.vy);
    }
  }
  // block reduction (warp shuffles, then one warp over the warp sums)
  __shared__ double red[4][32];
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = acc[k];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  const int nwarps = (blockDim.x * blockDim.y + 31) / 32;
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double v = lane < nwarps ? red[k][lane] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) partials[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * 4 + k] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Initial state f*_0 = f_eq(eps, u) (procedure item 1); NULL fields mean eps0 at rest.
// ---------------------------------------------------------------------------
template <typename S, int VS>
__global__ void init_kernel(S *__restrict__ fout, const Geometry<typename RealOf<S>::type> g, double eps0,
                            const double *__restrict__ eps, const double *__restrict__ ux,
                            const double *__restrict__ uy) {
  using V = VSet<VS>;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const long long c = (long long)y * g.nx + x;
  const double e = eps ? eps[c] / eps0 : 1.0;
  const double ax = ux ? ux[c] : 0.0, ay = uy ? uy[c] : 0.0;
  const double u2 = ax * ax + ay * ay, u0 = sqrt(1.0 + u2);
  const bool solid = g.nbmask && (g.nbmask[c] & 16u);
#pragma unroll
  for (int q = 0; q < V::Q; ++q) {
    const double uv = ax * V::vx(q) + ay * V::vy(q);
    const double heq = (e - 1.0) + V::CA * e * u0 * uv + V::CB * e * uv * uv - V::CC * e * u2;
    fout[q * g.plane + (long long)y * g.pitch + x] = store_h<S, typename RealOf<S>::type>(
        (typename RealOf<S>::type)(solid ? 0.0 : heq));
  }
}

// Stirring pipeline start at step n: coefficients of steps n and n+1, table of step n.
template <typename R>
__global__ void stir_draw_kernel(R4<R> *coef_a, R4<R> *coef_b, int nmodes, unsigned long long seed,
                                 long long n, double amp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nmodes) return;
  const int m = t % nmodes;
  double c[4];
  stir_draw(seed, n + t / nmodes, m, amp, c);
  (t < nmodes ? coef_a : coef_b)[m] = R4<R>{(R)c[0], (R)c[1], (R)c[2], (R)c[3]};
}

template <typename R>
__global__ void stir_table_kernel(const Stir<R> st, R4<R> *G, const R4<R> *coef, int nx) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)st.nrows * nx) return;
  G[t] = stir_row_entry<R>(st, coef, (int)(t / nx), (int)(t % nx), nx);
}

// ---------------------------------------------------------------------------
// Host launchers for this storage type
// ---------------------------------------------------------------------------
template <typename R> static Geometry<R> to_geom(const HostGeom &h) {
  Geometry<R> g;
  g.nx = h.nx; g.ny = h.ny; g.pitch = h.pitch; g.plane = h.plane; g.nbmask = h.nbmask;
  for (int q = 0; q < 17; ++q)
    for (int k = 0; k < 4; ++k) g.beta[q][k] = (R)h.beta[q][k];
  return g;
}

template <typename R> static Stir<R> to_stir(const HostStir &h) {
  Stir<R> s;
  s.nrows = h.nrows; s.nmodes = h.nmodes;
  s.G_cur = (const R4<R> *)h.G_cur; s.EY = (const R2<R> *)h.EY; s.G_next = (R4<R> *)h.G_next;
  s.coef_next = (const R4<R> *)h.coef_next; s.coef_new = (R4<R> *)h.coef_new;
  s.mode_kx = h.mode_kx; s.mode_ky = h.mode_ky; s.row_start = h.row_start; s.EX = (const R2<R> *)h.EX;
  s.seed = h.seed; s.step_new = h.step_new; s.amp = h.amp;
  return s;
}

template <typename S>
static cudaError_t launch_step_t(int vset, const void *fin, void *fout, const HostGeom &hg, const HostPhys &hp,
                                 const HostStir &hs, unsigned *err, dim3 block, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<R>(hg);
  Physics<R> p;
  p.omega0 = (R)hp.omega0; p.fpref = (R)hp.fpref; p.body_x = (R)hp.body_x; p.body_y = (R)hp.body_y;
  p.vmax2 = hp.vmax2; p.has_force = hp.has_force;
  const Stir<R> s = to_stir<R>(hs);
  const dim3 grid((hg.nx + block.x - 1) / block.x, (hg.ny + block.y - 1) / block.y);
  const bool mask = hg.nbmask != nullptr;
  const S *a = (const S *)fin;
  S *b = (S *)fout;
  if (vset == 3) {
    if (mask) step_kernel<S, 3, true><<<grid, block, 0, stream>>>(a, b, g, p, s, err);
    else step_kernel<S, 3, false><<<grid, block, 0, stream>>>(a, b, g, p, s, err);
  } else {
    if (mask) step_kernel<S, 2, true><<<grid, block, 0, stream>>>(a, b, g, p, s, err);
    else step_kernel<S, 2, false><<<grid, block, 0, stream>>>(a, b, g, p, s, err);
  }
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_moments_t(int vset, const void *fin, const HostGeom &hg, double eps0, double *eps,
                                    double *ux, double *uy, double *partials, unsigned *err, dim3 block,
                                    cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<R>(hg);
  const dim3 grid((hg.nx + block.x - 1) / block.x, (hg.ny + block.y - 1) / block.y);
  const bool mask = hg.nbmask != nullptr;
  const S *a = (const S *)fin;
  if (vset == 3) {
    if (mask) moments_kernel<S, 3, true><<<grid, block, 0, stream>>>(a, g, eps0, eps, ux, uy, partials, err);
    else moments_kernel<S, 3, false><<<grid, block, 0, stream>>>(a, g, eps0, eps, ux, uy, partials, err);
  } else {
    if (mask) moments_kernel<S, 2, true><<<grid, block, 0, stream>>>(a, g, eps0, eps, ux, uy, partials, err);
    else moments_kernel<S, 2, false><<<grid, block, 0, stream>>>(a, g, eps0, eps, ux, uy, partials, err);
  }
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_init_t(int vset, void *fout, const HostGeom &hg, double eps0, const double *eps,
                                 const double *ux, const double *uy, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<R>(hg);
  const dim3 block(32, 8);
  const dim3 grid((hg.nx + 31) / 32, (hg.ny + 7) / 8);
  if (vset == 3) init_kernel<S, 3><<<grid, block, 0, stream>>>((S *)fout, g, eps0, eps, ux, uy);
  else init_kernel<S, 2><<<grid, block, 0, stream>>>((S *)fout, g, eps0, eps, ux, uy);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_stir_prime_t(const HostStir &hs, void *coef_n, void *coef_n1, void *G_n, int nx,
                                       long long n, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  if (hs.nmodes == 0) return cudaSuccess;
  const Stir<R> s = to_stir<R>(hs);
  stir_draw_kernel<R><<<(2 * hs.nmodes + 127) / 128, 128, 0, stream>>>((R4<R> *)coef_n, (R4<R> *)coef_n1,
                                                                        hs.nmodes, hs.seed, n, hs.amp);
  const long long entries = (long long)hs.nrows * nx;
  stir_table_kernel<R><<<(unsigned)((entries + 255) / 256), 256, 0, stream>>>(s, (R4<R> *)G_n,
                                                                             (const R4<R> *)coef_n, nx);
  return cudaGetLastError();
}

}  // namespace rlbm

#define RLBM_CAT2(a, b) a##b
#define RLBM_CAT(a, b) RLBM_CAT2(a, b)
#define RLBM_DEFINE_LAUNCHERS(S, SUF)                                                                    \
  namespace rlbm {                                                                                       \
  cudaError_t RLBM_CAT(launch_step_, SUF)(int vset, const void *fin, void *fout, const HostGeom &g,     \
                                          const HostPhys &p, const HostStir &s, unsigned *err, dim3 b,  \
                                          cudaStream_t st) {                                             \
    return launch_step_t<S>(vset, fin, fout, g, p, s, err, b, st);                                       \
  }                                                                                                      \
  cudaError_t RLBM_CAT(launch_moments_, SUF)(int vset, const void *fin, const HostGeom &g, double eps0, \
                                             double *e, double *ux, double *uy, double *part,           \
                                             unsigned *err, dim3 b, cudaStream_t st) {                   \
    return launch_moments_t<S>(vset, fin, g, eps0, e, ux, uy, part, err, b, st);                         \
  }                                                                                                      \
  cudaError_t RLBM_CAT(launch_init_, SUF)(int vset, void *fout, const HostGeom &g, double eps0,         \
                                          const double *e, const double *ux, const double *uy,          \
                                          cudaStream_t st) {                                             \
    return launch_init_t<S>(vset, fout, g, eps0, e, ux, uy, st);                                         \
  }                                                                                                      \
  cudaError_t RLBM_CAT(launch_stir_prime_, SUF)(const HostStir &s, void *cn, void *cn1, void *G, int nx, \
                                                long long n, cudaStream_t st) {                          \
    return launch_stir_prime_t<S>(s, cn, cn1, G, nx, n, st);                                             \
  }                                                                                                      \
  }
