// Adjoint of the fused step: the gradient of a kinetic-energy objective of a stirred
// run with respect to the per-mode stirring multipliers sigma_m, eta/s and the body
// force, by reverse-mode differentiation written out by hand.
//
// With the post-collision buffer B_{n-1} of the forward run, S_n = P B_{n-1} (pull
// streaming) and B_n = C_n(S_n) (moments, Landau matching, equilibrium, Anderson-Witting
// relaxation and projected force of one cell), the adjoint kappa_n = dJ/dS_n obeys
//
//   kappa_n = dj_n/dS_n + (dC_n/dS)^T (P^T kappa_{n+1}),
//
// and every step adds (dC_n/dtheta)^T (P^T kappa_{n+1}) to the parameter gradients.
// One launch per step gathers S_n (forward pull of B_{n-1}) and P^T kappa_{n+1} (the
// transposed pull: reversed offsets, same bilinear weights, and at a solid corner the
// cell's own reversed plane, so it has the form of the forward pull), runs the cell's
// reverse and writes kappa_n.  Landau matching R(v) = m - T v - (T^00 - m.v) v = 0 is
// differentiated implicitly: the adjoint w solves (dR/dv)^T w = vbar and the moments
// receive -(dR/dp)^T w.  The recomputed forward of a segment keeps each step's Landau
// solution (eps - 1, v) and force (F_x, F_y) per cell; the reverse step reads them instead
// of solving Landau matching and synthesising the stirring force again (the force
// adjoint's row projections still use the step's tables).
#include "rlbm_kernels.cuh"

namespace rlbm {

template <typename R> struct AdjStir {
  int nrows;
  const R4<R> *G;    // [nrows][nx] table of the step (Gx.re, Gx.im, Gy.re, Gy.im)
  const R2<R> *EY;   // [nrows][eyp] exp(i 2 pi k_y y / ny)
  int eyp;
};

// Pulls of one cell from staged tiles (32 x 8 tile with its one-cell halo, the layout of
// the forward step kernel's stages; b0 = the cell's offset in a staged plane).
//   forward pull   h_q(x)   = sum_c beta_{q,c} B_q(x - o_c)
//   transposed     lam_q(x) = sum_c beta_{q,c} kappa_q(x + o_c)
// with o_c in {(0,0), (sx,0), (0,sy), (sx,sy)}.  A solid source corner of the forward pull
// takes the cell's own reversed plane B_{opp(q)}(x); in the transpose the same corner (the
// neighbour x + o_c) takes kappa_{opp(q)}(x).
template <typename T, int VS, bool MASK, int SIGN>
__device__ __forceinline__ void pull_staged(const T *tile, int plane, int txb, int b0, const Geometry<T> &g,
                                            unsigned nb, T out[VSet<VS>::Q]) {
  constexpr int Q = VSet<VS>::Q;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const T *pl = tile + q * plane + b0;
    const T *own = tile + VSet<VS>::opp(q) * plane + b0;
    const int sx = sgnx<VS>(q), sy = sgny<VS>(q);
    T acc = g.beta[q][0] * pl[0];
    if (sx != 0) acc += g.beta[q][1] * ((MASK && ((nb >> (4 + SIGN * sx)) & 1u)) ? *own : pl[SIGN * sx]);
    if (sy != 0) acc += g.beta[q][2] * ((MASK && ((nb >> (4 + 3 * SIGN * sy)) & 1u)) ? *own : pl[SIGN * sy * txb]);
    if (sx != 0 && sy != 0)
      acc += g.beta[q][3] *
             ((MASK && ((nb >> (4 + SIGN * (3 * sy + sx))) & 1u)) ? *own : pl[SIGN * (sy * txb + sx)]);
    out[q] = acc;
  }
}

// The same two pulls for the two cells (x, y) and (x, y + 1) of a thread (db = the staged offset
// of the second cell), as packed FP32 pairs: the FP32 reverse step.
template <int VS, bool MASK, int SIGN>
__device__ __forceinline__ void pull_staged_pair(const float *tile, int plane, int txb, int b0, int db,
                                                 const Geometry<float> &g, unsigned nbA, unsigned nbB,
                                                 F2 out[VSet<VS>::Q]) {
  constexpr int Q = VSet<VS>::Q;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const float *pl = tile + q * plane + b0;
    const float *own = tile + VSet<VS>::opp(q) * plane + b0;
    const int sx = sgnx<VS>(q), sy = sgny<VS>(q);
    F2 acc = F2(g.beta2[q][0]) * F2(pl[0], pl[db]);
    if (sx != 0) {
      float vA = pl[SIGN * sx], vB = pl[db + SIGN * sx];
      if (MASK && ((nbA >> (4 + SIGN * sx)) & 1u)) vA = own[0];
      if (MASK && ((nbB >> (4 + SIGN * sx)) & 1u)) vB = own[db];
      acc = fma(F2(g.beta2[q][1]), F2(vA, vB), acc);
    }
    if (sy != 0) {
      float vA = pl[SIGN * sy * txb], vB = pl[db + SIGN * sy * txb];
      if (MASK && ((nbA >> (4 + 3 * SIGN * sy)) & 1u)) vA = own[0];
      if (MASK && ((nbB >> (4 + 3 * SIGN * sy)) & 1u)) vB = own[db];
      acc = fma(F2(g.beta2[q][2]), F2(vA, vB), acc);
    }
    if (sx != 0 && sy != 0) {
      float vA = pl[SIGN * (sy * txb + sx)], vB = pl[db + SIGN * (sy * txb + sx)];
      if (MASK && ((nbA >> (4 + SIGN * (3 * sy + sx))) & 1u)) vA = own[0];
      if (MASK && ((nbB >> (4 + SIGN * (3 * sy + sx))) & 1u)) vB = own[db];
      acc = fma(F2(g.beta2[q][3]), F2(vA, vB), acc);
    }
    out[q] = acc;
  }
}

// Reverse of one cell's collision and force (coll_coeffs / collide_all) and of its
// objective term cj |v|^2 / 2, given the cell's post-streaming deviations h, their
// moments M and Landau solution m, and the adjoint lam of the cell's output.  Returns
// the adjoint of h in kap, d/d(ln omega0) in gom and the adjoint of F in gFx, gFy.
template <typename R, int VS, bool FORCE>
__device__ __forceinline__ void cell_adjoint(const R h[VSet<VS>::Q], const R lam[VSet<VS>::Q], const Mom<R> &M,
                                             const Macro<R> &m, R omega0, R fpref, R Fx, R Fy, R cj,
                                             R kap[VSet<VS>::Q], R &gom, R &gFx, R &gFy) {
  using V = VSet<VS>;
  constexpr int Q = V::Q;
  const R epsh = R(1) + m.eps_m1;
  const R om = VS == 3 ? omega0 * FM<R>::qroot(epsh) : omega0 * FM<R>::croot(epsh);
  const R u0 = m.u0, ux = m.ux, uy = m.uy;
  const R u2 = ux * ux + uy * uy;
  const R ca = R(V::CA) * epsh * u0, cb = R(V::CB) * epsh, cc = m.eps_m1 - R(V::CC) * epsh * u2;
  const R p1 = om * (u0 * ca - cc), p2 = om * (u0 * cb - ca), p3 = -om * cb;
  const R k0 = R(1) - om * u0;

  // h*_q = h_q (k0 + om t_q) + p0 + p1 t + p2 t^2 + p3 t^3 + S_q,  t_q = u . v_q
  R om_b = R(0), u0_b = R(0), ux_b = R(0), uy_b = R(0);
  R P0 = R(0), P1 = R(0), P2 = R(0), P3 = R(0);
  R S1x = R(0), S1y = R(0), Sxx = R(0), Sxy = R(0), Syy = R(0), Szz = R(0);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const R vx = R(V::vx(q)), vy = R(V::vy(q));
    const R t = ux * vx + uy * vy;
    const R lq = lam[q];
    kap[q] = lq * (k0 + om * t);
    const R lh = lq * h[q];
    om_b += lh * (t - u0);
    u0_b -= om * lh;
    const R tb = om * lh + lq * (p1 + t * (R(2) * p2 + R(3) * p3 * t));
    ux_b += tb * vx;
    uy_b += tb * vy;
    P0 += lq;
    P1 += lq * t;
    P2 += lq * t * t;
    P3 += lq * t * t * t;
    if (FORCE) {
      S1x += lq * vx;
      S1y += lq * vy;
      Sxx += lq * vx * vx;
      Sxy += lq * vx * vy;
      Syy += lq * vy * vy;
      Szz += lq * R(V::vz2(q));
    }
  }
  // p0 = om u0 cc, p1 = om (u0 ca - cc), p2 = om (u0 cb - ca), p3 = -om cb
  om_b += P0 * u0 * cc + P1 * (u0 * ca - cc) + P2 * (u0 * cb - ca) - P3 * cb;
  u0_b += om * (P0 * cc + P1 * ca + P2 * cb);
  const R cc_b = om * (P0 * u0 - P1);
  const R ca_b = om * (P1 * u0 - P2);
  const R cb_b = om * (P2 * u0 - P3);
  // ca = CA eps^ u0, cb = CB eps^, cc = (eps^ - 1) - CC eps^ |u|^2
  R epsh_b = ca_b * R(V::CA) * u0 + cb_b * R(V::CB) + cc_b * (R(1) - R(V::CC) * u2);
  u0_b += ca_b * R(V::CA) * epsh;
  ux_b -= cc_b * R(2 * V::CC) * epsh * ux;
  uy_b -= cc_b * R(2 * V::CC) * epsh * uy;
  // om = omega0 eps^(1/4) (D_p = 3) or omega0 eps^(1/3) (D_p = 2)
  epsh_b += divide(om_b * om, R(VS == 3 ? 4 : 3) * epsh);
  gom = om_b * om;

  R e_b = R(0), mx_b = R(0), my_b = R(0), txx_b = R(0), txy_b = R(0), tyy_b = R(0);
  R wxxx_b = R(0), wxxy_b = R(0), wxyy_b = R(0), wyyy_b = R(0);
  gFx = R(0);
  gFy = R(0);
  if (FORCE) {
    // s0 = fpref F.m / 4;  s1 = -fpref (1 + e) F / 2;  quadratic form with B and F m^T
    const R M0 = R(1) + M.e;
    const R f54 = R(1.25) * fpref;
    R FM1_b = R(0.25) * fpref * P0;
    e_b += R(-0.5) * fpref * (Fx * S1x + Fy * S1y);
    gFx += R(-0.5) * fpref * M0 * S1x;
    gFy += R(-0.5) * fpref * M0 * S1y;
    R Bxx_b = f54 * Sxx, Bxy_b = R(2) * f54 * Sxy, Byy_b = f54 * Syy;
    gFx -= R(2) * f54 * (M.mx * Sxx + M.my * Sxy);
    gFy -= R(2) * f54 * (M.mx * Sxy + M.my * Syy);
    mx_b -= R(2) * f54 * (Fx * Sxx + Fy * Sxy);
    my_b -= R(2) * f54 * (Fx * Sxy + Fy * Syy);
    // szz = f54 Bzz, Bzz = F.m - Bxx - Byy
    const R Bzz_b = f54 * Szz;
    FM1_b += Bzz_b;
    Bxx_b -= Bzz_b;
    Byy_b -= Bzz_b;
    // Bxx = Fx wxxx + Fy wxxy, Bxy = Fx wxxy + Fy wxyy, Byy = Fx wxyy + Fy wyyy
    gFx += Bxx_b * M.wxxx + Bxy_b * M.wxxy + Byy_b * M.wxyy;
    gFy += Bxx_b * M.wxxy + Bxy_b * M.wxyy + Byy_b * M.wyyy;
    wxxx_b += Bxx_b * Fx;
    wxxy_b += Bxx_b * Fy + Bxy_b * Fx;
    wxyy_b += Bxy_b * Fy + Byy_b * Fx;
    wyyy_b += Byy_b * Fy;
    gFx += FM1_b * M.mx;
    gFy += FM1_b * M.my;
    mx_b += FM1_b * Fx;
    my_b += FM1_b * Fy;
  }

  // objective and the macroscopic map: u0 = gamma, u = gamma v, eps^ = 1 + e - m.v
  const R vx = m.vx, vy = m.vy;
  R vx_b = cj * vx, vy_b = cj * vy;
  const R gam = u0;
  const R gam_b = u0_b + ux_b * vx + uy_b * vy;
  vx_b += ux_b * gam;
  vy_b += uy_b * gam;
  const R g3 = gam * gam * gam;
  vx_b += gam_b * g3 * vx;
  vy_b += gam_b * g3 * vy;
  e_b += epsh_b;
  mx_b -= epsh_b * vx;
  my_b -= epsh_b * vy;
  vx_b -= epsh_b * M.mx;
  vy_b -= epsh_b * M.my;

  // Landau: J = dR/dv = -T + v m^T - eps^ I;  J^T w = vbar;  pbar -= (dR/dp)^T w
  const R dinv = R(1.0 / V::DP);
  const R Txx = dinv + M.txx, Txy = M.txy, Tyy = dinv + M.tyy;
  const R jxx = -Txx + vx * M.mx - epsh, jxy = -Txy + vx * M.my;
  const R jyx = -Txy + vy * M.mx, jyy = -Tyy + vy * M.my - epsh;
  const R idet = divide(R(1), jxx * jyy - jxy * jyx);
  const R wx = (jyy * vx_b - jyx * vy_b) * idet;
  const R wy = (jxx * vy_b - jxy * vx_b) * idet;
  const R wv = wx * vx + wy * vy;
  e_b += wv;
  mx_b -= wx + vx * wv;
  my_b -= wy + vy * wv;
  txx_b += wx * vx;
  tyy_b += wy * vy;
  txy_b += wx * vy + wy * vx;

  // moments: e = sum w h, m = sum w h v, t = sum w h v v, third moments sum w h v v v
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const double qx = V::vx(q), qy = V::vy(q);
    R a = e_b;
    if (qx != 0.0) a += mx_b * R(qx) + txx_b * R(qx * qx);
    if (qy != 0.0) a += my_b * R(qy) + tyy_b * R(qy * qy);
    if (qx != 0.0 && qy != 0.0) a += txy_b * R(qx * qy);
    if (FORCE) {
      if (qx != 0.0) a += wxxx_b * R(qx * qx * qx);
      if (qx != 0.0 && qy != 0.0) a += wxxy_b * R(qx * qx * qy) + wxyy_b * R(qx * qy * qy);
      if (qy != 0.0) a += wyyy_b * R(qy * qy * qy);
    }
    kap[q] += R(V::w(q)) * a;
  }
}

// One adjoint step over the lattice.  Persistent CTAs of 256 threads (one cell each) walk
// the 32 x 8 tiles (tile t to CTA t mod grid); per tile one TMA box stages kappa_{n+1} (LAM)
// or, for the last state, B_{n-1}, with its one-cell halo, two stages rotating on mbarriers
// with bounded waits, as in the forward step kernel.
//   tB    load map of the post-collision buffer B_{n-1} of the forward run (used when LAM is
//         false: the last state, objective only, whose h is pulled and matched here)
//   tK    load map of kappa_{n+1} (LAM)
//   kout  kappa_n; ghost cells are written like the forward's (periodic copies)
//   cj    objective weight of S_n (1 / (N N_fluid), or 0 for the first state)
//   acc   per-tile FP64 sums, accumulated over steps: d/d(ln omega0), F adjoint x, y, J
//   zpart per tile row and k_y row r: sum over the tile's 8 rows of gF(x, y) EY_r(y)
//   macro (LAM) the step's eps/eps0 - 1, v_x, v_y, F_x, F_y and streamed h per cell (5 + Q
//         planes of nx * ny) as the forward step kernel computed them when it recomputed the
//         step; without LAM, Landau matching and the force synthesis are done here
template <typename S, int VS, bool MASK, bool FORCE, bool LAM, int NST>
__global__ void __launch_bounds__(256)
adjoint_kernel(const __grid_constant__ CUtensorMap tB, const __grid_constant__ CUtensorMap tK,
               typename RealOf<S>::type *__restrict__ kout, const Geometry<typename RealOf<S>::type> g,
               const Physics<typename RealOf<S>::type> p, const AdjStir<typename RealOf<S>::type> st,
               const typename RealOf<S>::type cj, double *__restrict__ acc, R4<typename RealOf<S>::type> *__restrict__ zpart,
               unsigned *__restrict__ err, const typename RealOf<S>::type *__restrict__ macro) {
  using R = typename RealOf<S>::type;
  using TL = Tile<S, VS>;
  static_assert(sizeof(S) == sizeof(R), "the adjoint runs on FP32 or FP64 storage");
  constexpr int Q = VSet<VS>::Q;
  constexpr int PL = TL::TYB * TL::TXB;  // elements of a staged plane
  constexpr int STAGE = TL::IN_STRIDE;  // kappa_{n+1} (LAM) or B_{n-1}
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + NST * STAGE);
  __shared__ R2<R> sF[8][32];
  __shared__ R2<R> sE[32][8];  // the tile's phase rows EY_r(y0 + j) of the force adjoint's projections
  __shared__ double red[8][4];
  const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5, lane = tid & 31, warp = tid >> 5;
  const int wid = blockIdx.x, nworkers = gridDim.x;
  const int ntx = (g.nx + 31) / 32, ntiles = ntx * ((g.ny + 7) / 8);
  const int my_tiles = wid < ntiles ? (ntiles - 1 - wid) / nworkers + 1 : 0;
  const uint32_t stage_bytes = TL::IN_BYTES;
  if (tid == 0) {
    for (int s2 = 0; s2 < NST; ++s2) mbar_init(&bar[s2], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0: the k-th tile of this CTA into stage k % NST (B, then kappa, on one barrier)
  auto issue_B = [&](int k) {
    if (LAM) return;
    const int t = wid + k * nworkers;
    const int x0 = (t % ntx) * TILE_X, y0 = (t / ntx) * TILE_Y;
    uint64_t *b = &bar[k % NST];
    mbar_expect_tx(b, stage_bytes);
    tma_load_3d(smem + (k % NST) * STAGE, &tB, b, x0 + TL::XOFF - TL::V, y0, 0);
  };
  auto issue_K = [&](int k) {
    if (!LAM) return;
    const int t = wid + k * nworkers;
    const int x0 = (t % ntx) * TILE_X, y0 = (t / ntx) * TILE_Y;
    uint64_t *b = &bar[k % NST];
    mbar_expect_tx(b, stage_bytes);
    tma_load_3d(smem + (k % NST) * STAGE, &tK, b, x0 + TL::XOFF - TL::V, y0, 0);
  };
  auto issue = [&](int k) { issue_B(k); issue_K(k); };
  // B_{n-1} (the last state) was written before the reverse sweep began, so its first tiles
  // are copied at once; a launch chained to the previous reverse step (programmatic
  // dependent launch) waits for that step's kappa_{n+1}, and writes nothing before.
  if (tid == 0)
    for (int k = 0; k < NST && k < my_tiles; ++k) issue_B(k);
  griddep_wait();
  if (tid == 0)
    for (int k = 0; k < NST && k < my_tiles; ++k) issue_K(k);
  bool alive = true;
  {
    const bool ok = my_tiles == 0 || mbar_wait_bounded(&bar[0], 0, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) alive = false;
  }
  for (int k = 0; alive && k < my_tiles; ++k) {
    // the next reverse step's grid may be scheduled once every CTA is on its last tile
    if (tid == 0 && k == my_tiles - 1) griddep_launch_dependents();
    const int t = wid + k * nworkers;
    const int tx = t % ntx, ty = t / ntx;
    const int x = tx * TILE_X + lx, y = ty * TILE_Y + ly;
    const S *tileB = reinterpret_cast<const S *>(smem + (k % NST) * STAGE);  // without LAM
    const R *tileK = reinterpret_cast<const R *>(smem + (k % NST) * STAGE);  // LAM
    const int b0 = (ly + 1) * TL::TXB + lx + TL::V;
    const bool inside = x < g.nx && y < g.ny;
    unsigned nb = 0;
    if (MASK && inside) nb = g.nbmask[(long long)y * g.nx + x];
    const bool fluid = inside && !(MASK && (nb & 16u));
    R kap[Q];
    R gom = R(0), gFx = R(0), gFy = R(0), jv = R(0);
#pragma unroll
    for (int q = 0; q < Q; ++q) kap[q] = R(0);
    // phase rows of the projections below, loaded now (one entry per thread: k_y row tid / 8,
    // tile row tid % 8) so that the loads complete while the cell's reverse runs
    R2<R> eyv{R(0), R(0)};
    const bool ey_shared = st.nrows <= 32;  // wider shells read the phase rows from global memory below
    const bool ey_loader = FORCE && ey_shared && tid < st.nrows * 8;
    if (ey_loader && ty * TILE_Y + (tid & 7) < g.ny)
      eyv = ey_at<R>(reinterpret_cast<const R *>(st.EY) + (long long)(tid >> 3) * 2 * st.eyp, ty * TILE_Y + (tid & 7));
    if (fluid) {
      R h[Q], lam[Q];
      // the forward's Landau solution, force and streamed h of this cell, loaded first so
      // that the loads overlap the pull
      R mv[5] = {R(0), R(0), R(0), R(0), R(0)};
      if (LAM) {
        const long long nc = (long long)g.nx * g.ny, c = (long long)y * g.nx + x;
#pragma unroll
        for (int k = 0; k < 5; ++k) mv[k] = macro[k * nc + c];
#pragma unroll
        for (int q = 0; q < Q; ++q) h[q] = macro[(5 + q) * nc + c];
        pull_staged<R, VS, MASK, 1>(tileK, PL, TL::TXB, b0, g, nb, lam);
      } else {
        pull_staged<R, VS, MASK, -1>(reinterpret_cast<const R *>(tileB), PL, TL::TXB, b0, g, nb, h);
#pragma unroll
        for (int q = 0; q < Q; ++q) lam[q] = R(0);
      }
      const Mom<R> M = moments_of<R, R, VS, FORCE>(h);
      Macro<R> m;
      R Fx = p.body_x, Fy = p.body_y;
      if (LAM) {
        // u^mu = gamma (1, v) as the step kernel forms it from v
        const R gam = FM<R>::rsqrt(R(1) - fma(mv[1], mv[1], mv[2] * mv[2]));
        m.eps_m1 = mv[0];
        m.vx = mv[1];
        m.vy = mv[2];
        m.u0 = gam;
        m.ux = gam * mv[1];
        m.uy = gam * mv[2];
        m.ok = true;
        Fx = mv[3];
        Fy = mv[4];
      } else {
        m = cell_macro<R, VS>(h, M, p.vmax2);
        if (!m.ok) atomicOr(err, (R(1) + m.eps_m1 > R(0) && isfinite(m.eps_m1)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
      }
      if (FORCE && !LAM) {
        // two rows per iteration, in two partial sums: both rows' loads are in flight at once
        const R *ey = reinterpret_cast<const R *>(st.EY);
        R Fx2 = R(0), Fy2 = R(0);
        int r = 0;
        for (; r + 1 < st.nrows; r += 2) {
          const R4<R> G0 = st.G[(long long)r * g.nx + x], G1 = st.G[(long long)(r + 1) * g.nx + x];
          const R2<R> E0 = ey_at<R>(ey + (long long)r * 2 * st.eyp, y);
          const R2<R> E1 = ey_at<R>(ey + (long long)(r + 1) * 2 * st.eyp, y);
          Fx = fma(G0.x, E0.x, fma(-G0.y, E0.y, Fx));
          Fy = fma(G0.z, E0.x, fma(-G0.w, E0.y, Fy));
          Fx2 = fma(G1.x, E1.x, fma(-G1.y, E1.y, Fx2));
          Fy2 = fma(G1.z, E1.x, fma(-G1.w, E1.y, Fy2));
        }
        if (r < st.nrows) {
          const R4<R> G0 = st.G[(long long)r * g.nx + x];
          const R2<R> E0 = ey_at<R>(ey + (long long)r * 2 * st.eyp, y);
          Fx = fma(G0.x, E0.x, fma(-G0.y, E0.y, Fx));
          Fy = fma(G0.z, E0.x, fma(-G0.w, E0.y, Fy));
        }
        Fx += Fx2;
        Fy += Fy2;
      }
      cell_adjoint<R, VS, FORCE>(h, lam, M, m, p.omega0, p.fpref, Fx, Fy, cj, kap, gom, gFx, gFy);
      jv = cj * R(0.5) * (m.vx * m.vx + m.vy * m.vy);
    }
    if (inside) {
      R *o = kout + (long long)(y + 1) * g.pitch + x + PadLayout<R>::XOFF;
#pragma unroll
      for (int q = 0; q < Q; ++q) o[q * g.plane] = kap[q];
      const int gxv = ghost_col(x, g.nx, g.walls);
      const int gyv = ghost_row(y, g.ny, g.walls);
      if (gxv != INT_MIN || gyv != INT_MIN) {
        const int px[3] = {gxv, x, gxv}, py[3] = {y, gyv, gyv};
        for (int a = 0; a < 3; ++a) {
          if (px[a] == INT_MIN || py[a] == INT_MIN) continue;
          R *d = kout + (long long)(py[a] + 1) * g.pitch + px[a] + PadLayout<R>::XOFF;
#pragma unroll
          for (int q = 0; q < Q; ++q) d[q * g.plane] = kap[q];
        }
      }
    }
    // projections of the force adjoint on the k_y rows of the stirring tables
    if (FORCE && st.nrows > 0) {
      sF[ly][lx] = R2<R>{gFx, gFy};
      if (ey_loader) sE[tid >> 3][tid & 7] = eyv;
      __syncthreads();
      const int jmax = g.ny - ty * TILE_Y;  // rows of this tile inside the lattice (>= 1)
      for (int r = ly; r < st.nrows; r += 8) {
        R4<R> z{R(0), R(0), R(0), R(0)};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (j < jmax) {
            const R2<R> E = ey_shared ? sE[r][j]
                                      : ey_at<R>(reinterpret_cast<const R *>(st.EY) + (long long)r * 2 * st.eyp,
                                                 ty * TILE_Y + j);
            const R2<R> F = sF[j][lx];
            z.x += F.x * E.x;
            z.y += F.x * E.y;
            z.z += F.y * E.x;
            z.w += F.y * E.y;
          }
        }
        if (x < g.nx) zpart[((long long)ty * st.nrows + r) * g.nx + x] = z;
      }
    }
    // tile sums (fixed order) added to this tile's accumulators: warp sums in the compute
    // type (GB300's FP64 rate is 1/64 of FP32), the eight warp sums in FP64
    R v[4] = {gom, gFx, gFy, jv};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], off);
      if (lane == 0) red[warp][c] = (double)v[c];
    }
    __syncthreads();
    if (tid < 4) {
      double sum = 0.0;
      for (int w8 = 0; w8 < 8; ++w8) sum += red[w8][tid];
      // one update of this slot per launch, launches in stream order: the same sum as a
      // plain read-add-write, without waiting for the read
      atomicAdd(&acc[(long long)t * 4 + tid], sum);
    }
    if (NST == 1) {  // the only stage is free once every thread is done with it
      __syncthreads();
      if (tid == 0 && k + 1 < my_tiles) issue(k + 1);
    }
    const bool ok = k + 1 >= my_tiles || mbar_wait_bounded(&bar[(k + 1) % NST], ((k + 1) / NST) & 1, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) {  // (NST = 2: also the barrier after which this stage is free)
      alive = false;
      break;
    }
    if (NST >= 2 && tid == 0 && k + NST < my_tiles) issue(k + NST);
  }
  if (!alive && tid == 0) {
    // a staged copy did not land in time: latch the error and wait (bounded) once more
    // for this CTA's copies still in flight before returning
    atomicOr(err, ERR_TIMEOUT);
    for (int s2 = 0; s2 < NST; ++s2) mbar_wait_bounded(&bar[s2], 0, WAIT_CYCLES);
  }
}

// The FP32 reverse step with two cells per thread (128 threads): cells (x, y) and (x, y + 1) of
// the 32 x 8 tile, the pulls, moments, the cell's reverse and the objective on packed FP32
// pairs, as the forward step kernel computes its FP32 paths.  Tile walk, staging, chaining,
// stores, row projections and tile sums as in adjoint_kernel.
template <int VS, bool MASK, bool FORCE, bool LAM, int NST>
__global__ void __launch_bounds__(128)
adjoint_pair_kernel(const __grid_constant__ CUtensorMap tB, const __grid_constant__ CUtensorMap tK,
                    float *__restrict__ kout, const Geometry<float> g, const Physics<float> p,
                    const AdjStir<float> st, const float cj, double *__restrict__ acc,
                    R4<float> *__restrict__ zpart, unsigned *__restrict__ err, const float *__restrict__ macro) {
  using TL = Tile<float, VS>;
  using T = F2;
  constexpr int Q = VSet<VS>::Q;
  constexpr int PL = TL::TYB * TL::TXB;  // elements of a staged plane
  constexpr int STAGE = TL::IN_STRIDE;  // kappa_{n+1} (LAM) or B_{n-1}
  constexpr int DB = TL::TXB;  // staged offset of a thread's second cell (the next row)
  constexpr int NT = 128;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + NST * STAGE);
  __shared__ R2<float> sF[8][32];
  __shared__ __align__(16) R2<float> sE[32][8];  // the tile's phase rows EY_r(y0 + j) of the projections
  __shared__ double red[4][4];
  const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5, lane = tid & 31, warp = tid >> 5;
  const int wid = blockIdx.x, nworkers = gridDim.x;
  const int ntx = (g.nx + 31) / 32, ntiles = ntx * ((g.ny + 7) / 8);
  const int my_tiles = wid < ntiles ? (ntiles - 1 - wid) / nworkers + 1 : 0;
  const uint32_t stage_bytes = TL::IN_BYTES;
  if (tid == 0) {
    for (int s2 = 0; s2 < NST; ++s2) mbar_init(&bar[s2], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue_B = [&](int k) {
    if (LAM) return;
    const int t = wid + k * nworkers;
    const int x0 = (t % ntx) * TILE_X, y0 = (t / ntx) * TILE_Y;
    uint64_t *b = &bar[k % NST];
    mbar_expect_tx(b, stage_bytes);
    tma_load_3d(smem + (k % NST) * STAGE, &tB, b, x0 + TL::XOFF - TL::V, y0, 0);
  };
  auto issue_K = [&](int k) {
    if (!LAM) return;
    const int t = wid + k * nworkers;
    const int x0 = (t % ntx) * TILE_X, y0 = (t / ntx) * TILE_Y;
    uint64_t *b = &bar[k % NST];
    mbar_expect_tx(b, stage_bytes);
    tma_load_3d(smem + (k % NST) * STAGE, &tK, b, x0 + TL::XOFF - TL::V, y0, 0);
  };
  auto issue = [&](int k) { issue_B(k); issue_K(k); };
  if (tid == 0)
    for (int k = 0; k < NST && k < my_tiles; ++k) issue_B(k);
  griddep_wait();
  if (tid == 0)
    for (int k = 0; k < NST && k < my_tiles; ++k) issue_K(k);
  bool alive = true;
  {
    const bool ok = my_tiles == 0 || mbar_wait_bounded(&bar[0], 0, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) alive = false;
  }
  const bool ey_shared = st.nrows <= 32;  // wider shells read the phase rows from global memory below
  const int ney = (FORCE && ey_shared) ? st.nrows * 8 : 0;
  for (int k = 0; alive && k < my_tiles; ++k) {
    if (tid == 0 && k == my_tiles - 1) griddep_launch_dependents();
    const int t = wid + k * nworkers;
    const int tx = t % ntx, ty = t / ntx;
    const int x = tx * TILE_X + lx, yA = ty * TILE_Y + 2 * ly, yB = yA + 1;
    const float *tileB = reinterpret_cast<const float *>(smem + (k % NST) * STAGE);  // without LAM
    const float *tileK = reinterpret_cast<const float *>(smem + (k % NST) * STAGE);  // LAM
    const int b0 = (2 * ly + 1) * TL::TXB + lx + TL::V;
    const bool inA = x < g.nx && yA < g.ny, inB = x < g.nx && yB < g.ny;
    unsigned nbA = 0, nbB = 0;
    if (MASK) {
      if (inA) nbA = g.nbmask[(long long)yA * g.nx + x];
      if (inB) nbB = g.nbmask[(long long)yB * g.nx + x];
    }
    const bool flA = inA && !(MASK && (nbA & 16u)), flB = inB && !(MASK && (nbB & 16u));
    // phase rows of the projections below, loaded now (entries tid and tid + 128: k_y row e / 8,
    // tile row e % 8) so that the loads complete while the cells' reverse runs
    R2<float> ey0{0.0f, 0.0f}, ey1{0.0f, 0.0f};
    const int yj = ty * TILE_Y + (tid & 7);
    if (tid < ney && yj < g.ny)
      ey0 = ey_at<float>(reinterpret_cast<const float *>(st.EY) + (long long)(tid >> 3) * 2 * st.eyp, yj);
    if (tid + NT < ney && yj < g.ny)
      ey1 = ey_at<float>(reinterpret_cast<const float *>(st.EY) + (long long)((tid + NT) >> 3) * 2 * st.eyp, yj);
    T kap[Q];
    T gom(0.0f), gFx(0.0f), gFy(0.0f), jv(0.0f);
#pragma unroll
    for (int q = 0; q < Q; ++q) kap[q] = T(0.0f);
    if (flA || flB) {
      T h[Q], lam[Q];
      // the forward's Landau solution, force and streamed h of the two cells, loaded first
      // so that the loads overlap the pull
      float mA[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, mB[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
      if (LAM) {
        const long long nc = (long long)g.nx * g.ny, cA = (long long)yA * g.nx + x, cB = (long long)yB * g.nx + x;
        float hA[Q], hB[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) hA[q] = hB[q] = 0.0f;
        if (flA) {
#pragma unroll
          for (int j = 0; j < 5; ++j) mA[j] = macro[j * nc + cA];
#pragma unroll
          for (int q = 0; q < Q; ++q) hA[q] = macro[(5 + q) * nc + cA];
        }
        if (flB) {
#pragma unroll
          for (int j = 0; j < 5; ++j) mB[j] = macro[j * nc + cB];
#pragma unroll
          for (int q = 0; q < Q; ++q) hB[q] = macro[(5 + q) * nc + cB];
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) h[q] = T(hA[q], hB[q]);
        pull_staged_pair<VS, MASK, 1>(tileK, PL, TL::TXB, b0, DB, g, nbA, nbB, lam);
      } else {
        pull_staged_pair<VS, MASK, -1>(tileB, PL, TL::TXB, b0, DB, g, nbA, nbB, h);
#pragma unroll
        for (int q = 0; q < Q; ++q) lam[q] = T(0.0f);
      }
      if (!(flA && flB)) {  // a lane without fluid (outside the lattice or solid) works on the rest state
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          h[q] = T(flA ? h[q].v.x : 0.0f, flB ? h[q].v.y : 0.0f);
          lam[q] = T(flA ? lam[q].v.x : 0.0f, flB ? lam[q].v.y : 0.0f);
        }
      }
      const Mom<T> M = moments_of<T, T, VS, FORCE>(h);
      Macro<T> m;
      T Fx(p.body_x), Fy(p.body_y);
      if (LAM) {
        // u^mu = gamma (1, v) as the step kernel forms it from v
        const T vx(mA[1], mB[1]), vy(mA[2], mB[2]);
        const T gam = FM<T>::rsqrt(T(1.0f) - fma(vx, vx, vy * vy));
        m.eps_m1 = T(mA[0], mB[0]);
        m.vx = vx;
        m.vy = vy;
        m.u0 = gam;
        m.ux = gam * vx;
        m.uy = gam * vy;
        m.ok = true;
        Fx = T(mA[3], mB[3]);
        Fy = T(mA[4], mB[4]);
      } else {
        m = cell_macro_pair<VS>(h, M, p.vmax2);
        if (!m.ok) atomicOr(err, (isfinite(m.eps_m1.v.x) && isfinite(m.eps_m1.v.y)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
        // (without kappa_{n+1}, the state's force meets a zero adjoint: the body force stands in)
      }
      cell_adjoint<T, VS, FORCE>(h, lam, M, m, T(p.omega0), T(p.fpref), Fx, Fy, T(cj), kap, gom, gFx, gFy);
      jv = T(cj) * T(0.5f) * fma(m.vx, m.vx, m.vy * m.vy);
      if (!(flA && flB)) {
#pragma unroll
        for (int q = 0; q < Q; ++q) kap[q] = T(flA ? kap[q].v.x : 0.0f, flB ? kap[q].v.y : 0.0f);
        gom = T(flA ? gom.v.x : 0.0f, flB ? gom.v.y : 0.0f);
        gFx = T(flA ? gFx.v.x : 0.0f, flB ? gFx.v.y : 0.0f);
        gFy = T(flA ? gFy.v.x : 0.0f, flB ? gFy.v.y : 0.0f);
        jv = T(flA ? jv.v.x : 0.0f, flB ? jv.v.y : 0.0f);
      }
    }
#pragma unroll
    for (int ln = 0; ln < 2; ++ln) {
      const int y = ln ? yB : yA;
      if (!(ln ? inB : inA)) continue;
      float *o = kout + (long long)(y + 1) * g.pitch + x + PadLayout<float>::XOFF;
#pragma unroll
      for (int q = 0; q < Q; ++q) o[q * g.plane] = ln ? kap[q].v.y : kap[q].v.x;
      const int gxv = ghost_col(x, g.nx, g.walls);
      const int gyv = ghost_row(y, g.ny, g.walls);
      if (gxv != INT_MIN || gyv != INT_MIN) {
        const int px[3] = {gxv, x, gxv}, py[3] = {y, gyv, gyv};
        for (int a = 0; a < 3; ++a) {
          if (px[a] == INT_MIN || py[a] == INT_MIN) continue;
          float *d = kout + (long long)(py[a] + 1) * g.pitch + px[a] + PadLayout<float>::XOFF;
#pragma unroll
          for (int q = 0; q < Q; ++q) d[q * g.plane] = ln ? kap[q].v.y : kap[q].v.x;
        }
      }
    }
    // tile sums (fixed order): the two cells of a thread, warp sums in FP32, the four warp
    // sums in FP64; the warp sums go to shared memory with the projections' inputs, so that
    // one barrier serves both
    float v[4] = {gom.v.x + gom.v.y, gFx.v.x + gFx.v.y, gFy.v.x + gFy.v.y, jv.v.x + jv.v.y};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      for (int off = 16; off > 0; off >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], off);
      if (lane == 0) red[warp][c] = (double)v[c];
    }
    const bool proj = FORCE && st.nrows > 0;
    if (proj) {
      sF[2 * ly][lx] = R2<float>{gFx.v.x, gFy.v.x};
      sF[2 * ly + 1][lx] = R2<float>{gFx.v.y, gFy.v.y};
      if (tid < ney) sE[tid >> 3][tid & 7] = ey0;
      if (tid + NT < ney) sE[(tid + NT) >> 3][tid & 7] = ey1;
    }
    __syncthreads();
    if (tid < 4) {
      double sum = 0.0;
      for (int w4 = 0; w4 < NT / 32; ++w4) sum += red[w4][tid];
      atomicAdd(&acc[(long long)t * 4 + tid], sum);
    }
    // projections of the force adjoint on the k_y rows of the stirring tables: the column's
    // 8 values of gF loaded once, (x, y) and (z, w) of each row's sum on packed pairs
    if (proj) {
      const int jmax = g.ny - ty * TILE_Y;  // rows of this tile inside the lattice (>= 1)
      F2 Fx8[8], Fy8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const R2<float> F = sF[j][lx];
        Fx8[j] = F2(j < jmax ? F.x : 0.0f);
        Fy8[j] = F2(j < jmax ? F.y : 0.0f);
      }
      if (ey_shared) {
        // two rows per warp at a time, each row's sums in two halves (even and odd j), so that
        // four independent FMA chains of four run at once; the phase rows in 16-byte loads
        for (int r = warp; r < st.nrows; r += 2 * (NT / 32)) {
          const int r2 = r + NT / 32;
          const bool two = r2 < st.nrows;
          const int rb = two ? r2 : r;  // (a second row past the last computes nothing stored)
          F2 a0(0.0f), a1(0.0f), a2(0.0f), a3(0.0f), b0(0.0f), b1(0.0f), b2(0.0f), b3(0.0f);
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const float4 ea = *reinterpret_cast<const float4 *>(&sE[r][j]);
            const float4 eb = *reinterpret_cast<const float4 *>(&sE[rb][j]);
            a0 = fma(Fx8[j], F2(ea.x, ea.y), a0);
            a1 = fma(Fy8[j], F2(ea.x, ea.y), a1);
            a2 = fma(Fx8[j + 1], F2(ea.z, ea.w), a2);
            a3 = fma(Fy8[j + 1], F2(ea.z, ea.w), a3);
            b0 = fma(Fx8[j], F2(eb.x, eb.y), b0);
            b1 = fma(Fy8[j], F2(eb.x, eb.y), b1);
            b2 = fma(Fx8[j + 1], F2(eb.z, eb.w), b2);
            b3 = fma(Fy8[j + 1], F2(eb.z, eb.w), b3);
          }
          if (x < g.nx) {
            const F2 zxy = a0 + a2, zzw = a1 + a3;
            zpart[((long long)ty * st.nrows + r) * g.nx + x] = R4<float>{zxy.v.x, zxy.v.y, zzw.v.x, zzw.v.y};
            if (two) {
              const F2 uxy = b0 + b2, uzw = b1 + b3;
              zpart[((long long)ty * st.nrows + r2) * g.nx + x] = R4<float>{uxy.v.x, uxy.v.y, uzw.v.x, uzw.v.y};
            }
          }
        }
      } else {
        for (int r = warp; r < st.nrows; r += NT / 32) {
          F2 zxy(0.0f), zzw(0.0f);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const R2<float> E = j < jmax ? ey_at<float>(reinterpret_cast<const float *>(st.EY) +
                                                            (long long)r * 2 * st.eyp, ty * TILE_Y + j)
                                         : R2<float>{0.0f, 0.0f};
            const F2 e(E.x, E.y);
            zxy = fma(Fx8[j], e, zxy);
            zzw = fma(Fy8[j], e, zzw);
          }
          if (x < g.nx) zpart[((long long)ty * st.nrows + r) * g.nx + x] = R4<float>{zxy.v.x, zxy.v.y, zzw.v.x, zzw.v.y};
        }
      }
    }
    if (NST == 1) {  // the only stage is free once every thread is done with it
      __syncthreads();
      if (tid == 0 && k + 1 < my_tiles) issue(k + 1);
    }
    const bool ok = k + 1 >= my_tiles || mbar_wait_bounded(&bar[(k + 1) % NST], ((k + 1) / NST) & 1, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) {  // (NST = 2: also the barrier after which this stage is free)
      alive = false;
      break;
    }
    if (NST >= 2 && tid == 0 && k + NST < my_tiles) issue(k + NST);
  }
  if (!alive && tid == 0) {
    atomicOr(err, ERR_TIMEOUT);
    for (int s2 = 0; s2 < NST; ++s2) mbar_wait_bounded(&bar[s2], 0, WAIT_CYCLES);
  }
}

// zsum_j[r][x] = sum over block rows of zpart_j: the k_y-row transform of the force
// adjoint of step j of a segment at column x (blockIdx.z = j), in the compute type.
template <typename R>
__global__ void zsum_kernel(const R4<R> *__restrict__ zpart, int nby, int nrows, int nx, R4<R> *__restrict__ zsum) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const long long j = blockIdx.z;
  if (x >= nx) return;
  const R4<R> *zp = zpart + j * nby * nrows * nx + (long long)r * nx + x;
  R4<R> s{R(0), R(0), R(0), R(0)};
#pragma unroll 8
  for (int b = 0; b < nby; ++b) {
    const R4<R> z = zp[(long long)b * nrows * nx];
    s.x += z.x; s.y += z.y; s.z += z.z; s.w += z.w;
  }
  zsum[(j * nrows + r) * nx + x] = s;
}

constexpr int MG_THREADS = 128;        // threads of a mode-gradient block
constexpr int MG_MAX_ROW_MODES = 64;   // modes of one k_y row reduced per pass
static_assert(MG_MAX_ROW_MODES <= MG_THREADS, "one thread per mode finishes a pass");

// gstep[j][m] = d/d sigma_m of sum_x gF(x) . F(x) for the draws of step n0 + j
// (blockIdx.x = k_y row, blockIdx.y = j):
//   F(x, y) = sum_m sigma_m Re[(cx_m, cy_m) exp(i 2 pi (k_x x / nx + k_y y / ny))],
// so the derivative is Re[cx_m W_x] + Re[cy_m W_y] with W = sum_x exp(i 2 pi k_x x / nx) zsum_r(x).
// The per-step values are summed over all steps, in step order, at the end of the run,
// so the checkpoint segmentation does not change a bit.
template <typename R>
__global__ void __launch_bounds__(MG_THREADS)
mode_grad_kernel(const R4<R> *__restrict__ zsum, int nrows, const R2<R> *__restrict__ tw,
                 const int *__restrict__ mode_kx, const int *__restrict__ row_start, int nx,
                 unsigned long long seed, long long n0, double amp, int nmodes, double *__restrict__ gstep) {
  // one block per (k_y row r, step j): the row's transform is read from L2 for all its modes,
  // MG_MAX_ROW_MODES modes at a time
  const int r = blockIdx.x, j = blockIdx.y;
  const R4<R> *zs = zsum + ((long long)j * nrows + r) * nx;
  __shared__ double red[MG_MAX_ROW_MODES][MG_THREADS / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = row_start[r], m1 = row_start[r + 1]; c0 < m1; c0 += MG_MAX_ROW_MODES) {
    const int c1 = min(m1, c0 + MG_MAX_ROW_MODES);
    for (int mo = c0; mo < c1; ++mo) {
      const int kx = mode_kx[mo];
      R a[4] = {R(0), R(0), R(0), R(0)};
      for (int x = threadIdx.x; x < nx; x += MG_THREADS) {
        int t = (kx * x) % nx;
        if (t < 0) t += nx;
        const R2<R> e = tw[t];
        const R4<R> z = zs[x];
        a[0] += e.x * z.x - e.y * z.y;
        a[1] += e.x * z.y + e.y * z.x;
        a[2] += e.x * z.z - e.y * z.w;
        a[3] += e.x * z.w + e.y * z.z;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double v = (double)a[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[mo - c0][warp][k] = v;
      }
    }
    __syncthreads();
    // the draws of the step and the derivative: one thread per mode
    const int mo = c0 + (int)threadIdx.x;
    if (mo < c1) {
      double W[4] = {0.0, 0.0, 0.0, 0.0};
      for (int w = 0; w < MG_THREADS / 32; ++w)
        for (int k = 0; k < 4; ++k) W[k] += red[mo - c0][w][k];
      double c[4];
      if constexpr (sizeof(R) == 8) {
        stir_draw(seed, n0 + j, mo, amp, c);
      } else {
        float cf[4];
        stir_draw_f32(seed, n0 + j, mo, (float)amp, cf);
        for (int k = 0; k < 4; ++k) c[k] = (double)cf[k];
      }
      gstep[(long long)j * nmodes + mo] = c[0] * W[0] - c[1] * W[1] + c[2] * W[2] - c[3] * W[3];
    }
    __syncthreads();  // red is refilled by the next chunk
  }
}

// gsig[m] = sum over the run's steps n = 0 .. N-1 of gstep[n][m], in step order.
__global__ void mode_sum_kernel(const double *__restrict__ gstep, long long nsteps, int nmodes, double *__restrict__ gsig) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmodes) return;
  double s = 0.0;
  for (long long n = 0; n < nsteps; ++n) s += gstep[n * nmodes + m];
  gsig[m] = s;
}

// exp(+2 pi i t / n) for t < n, FP64 and rounded to FP32
__global__ void adj_twiddle_kernel(double2 *tw, float2 *twf, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double s, c;
  sincospi(2.0 * t / n, &s, &c);
  tw[t] = make_double2(c, s);
  twf[t] = make_float2((float)c, (float)s);
}

// The reverse-step kernel of a storage type (same parameters for both forms).
template <typename S, int VS, bool MASK, bool FORCE, bool LAM, int NST>
static auto pick_adjoint_kernel() {
  if constexpr (sizeof(S) == 4) return adjoint_pair_kernel<VS, MASK, FORCE, LAM, NST>;
  else return adjoint_kernel<S, VS, MASK, FORCE, LAM, NST>;
}

template <typename S, int VS, bool MASK, bool FORCE, bool LAM>
static cudaError_t launch_adjoint_k(const AdjointArgs &a, const Geometry<typename RealOf<S>::type> &g,
                                    const Physics<typename RealOf<S>::type> &p,
                                    const AdjStir<typename RealOf<S>::type> &s, cudaStream_t st) {
  // only a launch with kappa_{n+1} directly follows another reverse step
  using R = typename RealOf<S>::type;
  using TL = Tile<S, VS>;
  constexpr int NST = 2;
  // FP32: two cells per thread on packed pairs (128 threads); FP64: one cell per thread
  constexpr bool PAIR = sizeof(S) == 4;
  constexpr int NT = PAIR ? 128 : 256;
  auto kern = pick_adjoint_kernel<S, VS, MASK, FORCE, LAM, NST>();
  const int smem = NST * TL::IN_STRIDE + 64 + 128;
  static int configured_dev = -1, max_blocks = 0, sms = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_blocks, kern, NT, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    configured_dev = dev;
  }
  const int ntiles = ((g.nx + TILE_X - 1) / TILE_X) * ((g.ny + TILE_Y - 1) / TILE_Y);
  int workers = max_blocks * sms;
  if (workers > ntiles) workers = ntiles;
  if (workers < 1) workers = 1;
  const CUtensorMap &mB = *static_cast<const CUtensorMap *>(a.tB);
  const CUtensorMap &mK = LAM ? *static_cast<const CUtensorMap *>(a.tK) : mB;
  if (LAM && a.chained) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(workers);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, mB, mK, (R *)a.kout, g, p, s, (R)a.cj, a.acc, (R4<R> *)a.zpart, a.err,
                              (const R *)a.macro);
  }
  kern<<<workers, NT, smem, st>>>(mB, mK, (R *)a.kout, g, p, s, (R)a.cj, a.acc, (R4<R> *)a.zpart, a.err,
                                  (const R *)a.macro);
  return cudaGetLastError();
}

template <typename S, int VS, bool MASK, bool FORCE>
static cudaError_t launch_adjoint_v(const AdjointArgs &a, const Geometry<typename RealOf<S>::type> &g,
                                    const Physics<typename RealOf<S>::type> &p, cudaStream_t st) {
  using R = typename RealOf<S>::type;
  AdjStir<R> s;
  s.nrows = FORCE ? a.nrows : 0;
  s.G = (const R4<R> *)a.G;
  s.EY = (const R2<R> *)a.EY;
  s.eyp = a.eyp;
  if (a.kin) {
    if (!a.macro) return cudaErrorInvalidValue;  // a reverse step reads its forward step's stored values
    return launch_adjoint_k<S, VS, MASK, FORCE, true>(a, g, p, s, st);
  }
  return launch_adjoint_k<S, VS, MASK, FORCE, false>(a, g, p, s, st);
}

// dJ/dsigma contributions of nj consecutive steps n0 .. n0 + nj - 1 whose adjoint launches
// left their row projections in zpart[j] (j = n - n0).
template <typename R>
static cudaError_t launch_mode_grads_t(const ModeGradArgs &a, cudaStream_t st) {
  if (a.nrows == 0 || a.nmodes == 0 || a.nj == 0) return cudaSuccess;
  zsum_kernel<R><<<dim3((a.nx + 127) / 128, a.nrows, a.nj), 128, 0, st>>>((const R4<R> *)a.zpart, a.nby, a.nrows, a.nx,
                                                                         (R4<R> *)a.zsum);
  const void *tw = sizeof(R) == 8 ? a.tw : a.twf;
  mode_grad_kernel<R><<<dim3(a.nrows, a.nj), MG_THREADS, 0, st>>>((const R4<R> *)a.zsum, a.nrows, (const R2<R> *)tw,
                                                                  a.mode_kx, a.row_start, a.nx, a.seed, a.n0, a.amp,
                                                                  a.nmodes, a.gstep);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_adjoint_t(int vset, const AdjointArgs &a, const HostGeom &hg, const HostPhys &hp,
                                    cudaStream_t st) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<R>(hg);
  Physics<R> p{};
  p.omega0 = (R)hp.omega0; p.fpref = (R)hp.fpref; p.body_x = (R)hp.body_x; p.body_y = (R)hp.body_y;
  p.vmax2 = (R)hp.vmax2;
  const bool mask = hg.nbmask != nullptr, force = hp.has_force != 0;
  if (vset == 3) {
    if (force) {
      if (mask) return launch_adjoint_v<S, 3, true, true>(a, g, p, st);
      return launch_adjoint_v<S, 3, false, true>(a, g, p, st);
    }
    if (mask) return launch_adjoint_v<S, 3, true, false>(a, g, p, st);
    return launch_adjoint_v<S, 3, false, false>(a, g, p, st);
  }
  if (mask) return launch_adjoint_v<S, 2, true, false>(a, g, p, st);
  return launch_adjoint_v<S, 2, false, false>(a, g, p, st);
}

cudaError_t launch_adjoint_f64(int vset, const AdjointArgs &a, const HostGeom &g, const HostPhys &p, cudaStream_t st) {
  return launch_adjoint_t<double>(vset, a, g, p, st);
}
cudaError_t launch_adjoint_f32(int vset, const AdjointArgs &a, const HostGeom &g, const HostPhys &p, cudaStream_t st) {
  return launch_adjoint_t<float>(vset, a, g, p, st);
}
cudaError_t launch_mode_grads_f64(const ModeGradArgs &a, cudaStream_t st) { return launch_mode_grads_t<double>(a, st); }
cudaError_t launch_mode_grads_f32(const ModeGradArgs &a, cudaStream_t st) { return launch_mode_grads_t<float>(a, st); }
cudaError_t launch_mode_sum(const double *gstep, long long nsteps, int nmodes, double *gsig, cudaStream_t st) {
  if (nmodes == 0) return cudaSuccess;
  mode_sum_kernel<<<(nmodes + 127) / 128, 128, 0, st>>>(gstep, nsteps, nmodes, gsig);
  return cudaGetLastError();
}
cudaError_t launch_adj_twiddles(double2 *tw, float2 *twf, int n, cudaStream_t st) {
  adj_twiddle_kernel<<<(n + 255) / 256, 256, 0, st>>>(tw, twf, n);
  return cudaGetLastError();
}

}  // namespace rlbm
