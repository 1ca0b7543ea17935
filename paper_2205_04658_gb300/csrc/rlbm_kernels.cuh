// Kernels of the relativistic lattice Boltzmann update (arXiv 2205.04658) and the
// host launchers of one storage type.  Included once per storage type by
// rlbm_kernels_<type>.cu.
#pragma once

#include "rlbm_device.cuh"
#include "rlbm_launch.h"
#include "rlbm_tma.cuh"

#include <climits>
#include <type_traits>

namespace rlbm {

constexpr int TILE_X = 32, TILE_Y = 8, NTHREADS = TILE_X * TILE_Y;

// The ghost column a cell at x also writes (INT_MIN: none): with x periodic, its image
// beyond the opposite edge; in an open channel, the last column repeats itself beyond the
// outflow edge and nothing is written into the inflow column.
__device__ __forceinline__ int ghost_col(int x, int nx, int walls) {
  if (walls & OPEN_X) return x == nx - 1 ? nx : INT_MIN;
  return x == 0 ? nx : (x == nx - 1 ? -1 : INT_MIN);
}
__device__ __forceinline__ int ghost_row(int y, int ny, int walls) {
  return (walls & (WALLS_Y | STRIP_Y)) ? INT_MIN : (y == 0 ? ny : (y == ny - 1 ? -1 : INT_MIN));
}
constexpr long long WAIT_CYCLES = 4000000000ll;  // ~2 s at 2 GHz: bounded TMA waits

template <typename S, int VS> struct Tile {
  static constexpr int Q = VSet<VS>::Q;
  static constexpr int V = PadLayout<S>::V;
  static constexpr int XOFF = PadLayout<S>::XOFF;
  static constexpr int TXB = TILE_X + 2 * V;         // staged columns (16-byte granules on both sides)
  static constexpr int TYB = TILE_Y + 2;             // staged rows (one halo row each side)
  static constexpr int IN_BYTES = Q * TYB * TXB * (int)sizeof(S);
  static constexpr int IN_STRIDE = (IN_BYTES + 127) / 128 * 128;
  // stirring tables of the tile (at most MAX_SROWS k_y rows): G[row][TILE_X] (R4) and
  // EY[row][TILE_Y] (R2) after the populations; their size follows the shell at run time
  using R = typename RealOf<S>::type;
  static constexpr int MAX_SROWS = 16;
  static constexpr int G_ROW = TILE_X * 4 * (int)sizeof(R);
  static constexpr int EY_ROW = TILE_Y * 2 * (int)sizeof(R);
  static_assert(IN_STRIDE % 128 == 0 && G_ROW % 128 == 0, "TMA shared-memory destinations are 128-byte aligned");
  __host__ __device__ static constexpr int g_bytes(int rows) { return (rows * G_ROW + 127) / 128 * 128; }
  __host__ __device__ static constexpr int ey_bytes(int rows) { return (rows * EY_ROW + 127) / 128 * 128; }
  __host__ __device__ static constexpr int stage(int rows) { return IN_STRIDE + g_bytes(rows) + ey_bytes(rows); }
  __host__ __device__ static constexpr int smem(int nst, int rows) { return nst * stage(rows) + 64 + 128; }
};

// One cell per thread (256 threads): the FP64 path.
template <typename S, int VS, bool MASK, bool FORCE, int CPT, class G, class W>
__device__ __forceinline__ typename std::enable_if<CPT == 1>::type
tile_cells(const unsigned char *stg, int ey_off, S *fout, int x0, int y0, int tid, const G &g, const W &wts,
           const Physics<typename RealOf<S>::type> &p, const Stir<typename RealOf<S>::type> &st, bool staged,
           unsigned *err, typename RealOf<S>::type *macro_out) {
  using R = typename RealOf<S>::type;
  using V = VSet<VS>;
  using TL = Tile<S, VS>;
  constexpr int Q = V::Q;
    const int lx = tid % TILE_X, ly = tid / TILE_X;
    const int x = x0 + lx, y = y0 + ly;
    const S *tile = reinterpret_cast<const S *>(stg);
    const bool inside = x < g.nx && y < g.ny;
    unsigned nb = 0;
    if (MASK && g.nbmask && inside) nb = g.nbmask[(long long)y * g.nx + x];
    const bool fluid = inside && !(MASK && (nb & 16u));
    R hn[Q];
    if (fluid) {
      // pull-streaming from the staged tile: cell (lx, ly) at row ly + 1, column lx + V
      const int b0 = (ly + 1) * TL::TXB + lx + TL::V;
      R h[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const S *pl = tile + q * TL::TYB * TL::TXB + b0;
        const int sx = sgnx<VS>(q), sy = sgny<VS>(q);
        const R c = load_h_s<S, R>(pl);
        R acc = wts.beta[q][0] * c;
        if (sx != 0) {
          R v = load_h_s<S, R>(pl - sx);
          if (MASK && ((nb >> (4 - sx)) & 1u)) v = load_h_s<S, R>(tile + V::opp(q) * TL::TYB * TL::TXB + b0);
          acc = fma(wts.beta[q][1], v, acc);
        }
        if (sy != 0) {
          R v = load_h_s<S, R>(pl - sy * TL::TXB);
          if (MASK && ((nb >> (4 - 3 * sy)) & 1u)) v = load_h_s<S, R>(tile + V::opp(q) * TL::TYB * TL::TXB + b0);
          acc = fma(wts.beta[q][2], v, acc);
        }
        if (sx != 0 && sy != 0) {
          R v = load_h_s<S, R>(pl - sy * TL::TXB - sx);
          if (MASK && ((nb >> (4 - 3 * sy - sx)) & 1u)) v = load_h_s<S, R>(tile + V::opp(q) * TL::TYB * TL::TXB + b0);
          acc = fma(wts.beta[q][3], v, acc);
        }
        h[q] = acc;
      }
      const Mom<R> M = moments_of<R, R, VS, FORCE>(h);
      const Macro<R> m = cell_macro<R, VS>(h, M, p.vmax2);
      if (!m.ok) atomicOr(err, (R(1) + m.eps_m1 > R(0) && isfinite(m.eps_m1)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
      R Fx = p.body_x, Fy = p.body_y;
      if (FORCE) {
        if (staged) {
          const R4<R> *Gs = reinterpret_cast<const R4<R> *>(stg + TL::IN_STRIDE) + lx;
          const R *Er = reinterpret_cast<const R *>(stg + ey_off) + ey_index(ly);
          // F = sum_r Re[G_r(x) EY_r(y)], two rows per iteration (staged phase rows: 16 reals)
          R Fx2 = R(0), Fy2 = R(0);
          int r = 0;
#pragma unroll 1
          for (; r + 1 < st.nrows; r += 2) {
            const R4<R> G0 = Gs[r * TILE_X], G1 = Gs[(r + 1) * TILE_X];
            const R2<R> E0{Er[r * 16], Er[r * 16 + 2]}, E1{Er[(r + 1) * 16], Er[(r + 1) * 16 + 2]};
            Fx = fma(G0.x, E0.x, fma(-G0.y, E0.y, Fx));
            Fy = fma(G0.z, E0.x, fma(-G0.w, E0.y, Fy));
            Fx2 = fma(G1.x, E1.x, fma(-G1.y, E1.y, Fx2));
            Fy2 = fma(G1.z, E1.x, fma(-G1.w, E1.y, Fy2));
          }
          if (r < st.nrows) {
            const R4<R> G0 = Gs[r * TILE_X];
            const R2<R> E0{Er[r * 16], Er[r * 16 + 2]};
            Fx = fma(G0.x, E0.x, fma(-G0.y, E0.y, Fx));
            Fy = fma(G0.z, E0.x, fma(-G0.w, E0.y, Fy));
          }
          Fx += Fx2;
          Fy += Fy2;
        } else {
          for (int r = 0; r < st.nrows; ++r) {
            const R4<R> G = st.G_cur[(long long)r * g.nx + x];
            const R2<R> E = ey_at<R>(reinterpret_cast<const R *>(st.EY) + (long long)r * 2 * st.eyp, y);
            Fx += G.x * E.x - G.y * E.y;
            Fy += G.z * E.x - G.w * E.y;
          }
        }
      }
      if (macro_out) {  // the cell's Landau solution, force and streamed h, kept for the reverse sweep
        const long long nc = (long long)g.nx * g.ny, c = (long long)y * g.nx + x;
        macro_out[c] = m.eps_m1;
        macro_out[nc + c] = m.vx;
        macro_out[2 * nc + c] = m.vy;
        macro_out[3 * nc + c] = Fx;
        macro_out[4 * nc + c] = Fy;
#pragma unroll
        for (int q = 0; q < Q; ++q) macro_out[(5 + q) * nc + c] = h[q];
      }
      const Coll<R> cf = coll_coeffs<R, VS, FORCE>(M, m, p.omega0, p.fpref, Fx, Fy);
      collide_all<R, VS, FORCE>(cf, h, hn);
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) hn[q] = R(0);
    }
    if (inside) {  // coalesced stores straight from registers (one 128-byte line per warp and plane)
      S *o = fout + (long long)(y + 1) * g.pitch + x + TL::XOFF;
#pragma unroll
      for (int q = 0; q < Q; ++q) o[q * g.plane] = store_h<S, R>(hn[q]);
    }
    // ghost copies of the periodic neighbours (boundary cells only)
    if (inside) {
      const int gxv = ghost_col(x, g.nx, g.walls);
      const int gyv = ghost_row(y, g.ny, g.walls);
      if (gxv != INT_MIN || gyv != INT_MIN) {
        const int px[3] = {gxv, x, gxv}, py[3] = {y, gyv, gyv};
        for (int a = 0; a < 3; ++a) {
          if (px[a] == INT_MIN || py[a] == INT_MIN) continue;
          S *o = fout + (long long)(py[a] + 1) * g.pitch + px[a] + TL::XOFF;
#pragma unroll
          for (int q = 0; q < Q; ++q) o[q * g.plane] = store_h<S, R>(hn[q]);
        }
      }
    }
}

// Two cells per thread (128 threads): cells (x, y) and (x, y + 1) of the 32 x 8 tile (y
// even), all per-cell arithmetic on packed FP32 pairs.  The FP32, FP16 and BF16 paths.  The
// two cells are adjacent rows, so the classes that move in y pull one of their rows for
// both (each such value is read from shared memory and converted once).
template <typename S, int VS, bool MASK, bool FORCE, int CPT, class G, class W>
__device__ __forceinline__ typename std::enable_if<CPT == 2>::type
tile_cells(const unsigned char *stg, int ey_off, S *fout, int x0, int y0, int tid, const G &g, const W &wts,
           const Physics<float> &p, const Stir<float> &st, bool staged, unsigned *err, float *macro_out) {
  using V = VSet<VS>;
  using TL = Tile<S, VS>;
  using T = F2;
  constexpr int Q = V::Q;
  constexpr int DB = TL::TXB;  // smem offset of the second cell
  const int lx = tid % TILE_X, ly = tid / TILE_X;
  const int x = x0 + lx, yA = y0 + 2 * ly, yB = yA + 1;
  const S *tile = reinterpret_cast<const S *>(stg);
  const bool inA = x < g.nx && yA < g.ny, inB = x < g.nx && yB < g.ny;
  unsigned nbA = 0, nbB = 0;
  if (MASK && g.nbmask) {
    if (inA) nbA = g.nbmask[(long long)yA * g.nx + x];
    if (inB) nbB = g.nbmask[(long long)yB * g.nx + x];
  }
  const bool flA = inA && !(MASK && (nbA & 16u)), flB = inB && !(MASK && (nbB & 16u));
  const bool both = flA && flB;
  T hn[Q];
  if (flA || flB) {
    const int b0 = (2 * ly + 1) * TL::TXB + lx + TL::V;
    T h[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const S *pl = tile + q * TL::TYB * TL::TXB + b0;
      const S *own = tile + V::opp(q) * TL::TYB * TL::TXB + b0;
      const int sx = sgnx<VS>(q), sy = sgny<VS>(q);
      T acc = T(wts.beta2[q][0]) * T(load_s_raw<S>(pl), load_s_raw<S>(pl + DB));
      if (sx != 0) {
        float vA = load_s_raw<S>(pl - sx), vB = load_s_raw<S>(pl + DB - sx);
        if (MASK && ((nbA >> (4 - sx)) & 1u)) vA = load_s_raw<S>(own);
        if (MASK && ((nbB >> (4 - sx)) & 1u)) vB = load_s_raw<S>(own + DB);
        acc = fma(T(wts.beta2[q][1]), T(vA, vB), acc);
      }
      if (sy != 0) {
        float vA = load_s_raw<S>(pl - sy * TL::TXB), vB = load_s_raw<S>(pl + DB - sy * TL::TXB);
        if (MASK && ((nbA >> (4 - 3 * sy)) & 1u)) vA = load_s_raw<S>(own);
        if (MASK && ((nbB >> (4 - 3 * sy)) & 1u)) vB = load_s_raw<S>(own + DB);
        acc = fma(T(wts.beta2[q][2]), T(vA, vB), acc);
      }
      if (sx != 0 && sy != 0) {
        float vA = load_s_raw<S>(pl - sy * TL::TXB - sx), vB = load_s_raw<S>(pl + DB - sy * TL::TXB - sx);
        if (MASK && ((nbA >> (4 - 3 * sy - sx)) & 1u)) vA = load_s_raw<S>(own);
        if (MASK && ((nbB >> (4 - 3 * sy - sx)) & 1u)) vB = load_s_raw<S>(own + DB);
        acc = fma(T(wts.beta2[q][3]), T(vA, vB), acc);
      }
      h[q] = acc;
    }
    if (!both) {  // a lane without fluid (outside the lattice or solid) computes the rest state
#pragma unroll
      for (int q = 0; q < Q; ++q) h[q] = T(flA ? h[q].v.x : 0.0f, flB ? h[q].v.y : 0.0f);
    }
    const Mom<T> M = moments_of<T, T, VS, FORCE>(h);
    const Macro<T> m = cell_macro_pair<VS>(h, M, p.vmax2);
    if (!m.ok) atomicOr(err, (isfinite(m.eps_m1.v.x) && isfinite(m.eps_m1.v.y)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
    T Fx(p.body_x), Fy(p.body_y);
    if (FORCE) {
      if (staged) {
        const R4<float> *Gs = reinterpret_cast<const R4<float> *>(stg + TL::IN_STRIDE) + lx;
        // (Re yA, Re yB, Im yA, Im yB) of each staged phase row: the pairs load as they are used.
        // Two rows per iteration into two partial sums, so that both rows' loads and FMA chains
        // are in flight at once (the synthesis is latency-bound when it runs one row at a time).
        const R4<float> *Es = reinterpret_cast<const R4<float> *>(stg + ey_off) + ly;
        T Fx2(0.0f), Fy2(0.0f);
        int r = 0;
#pragma unroll 1
        for (; r + 1 < st.nrows; r += 2) {
          const R4<float> G = Gs[r * TILE_X], G1 = Gs[(r + 1) * TILE_X];
          const R4<float> E = Es[r * 4], E1 = Es[(r + 1) * 4];
          const T Ere(E.x, E.y), Eim(E.z, E.w), Ere1(E1.x, E1.y), Eim1(E1.z, E1.w);
          Fx = fma(T(G.x), Ere, fma(T(-G.y), Eim, Fx));
          Fy = fma(T(G.z), Ere, fma(T(-G.w), Eim, Fy));
          Fx2 = fma(T(G1.x), Ere1, fma(T(-G1.y), Eim1, Fx2));
          Fy2 = fma(T(G1.z), Ere1, fma(T(-G1.w), Eim1, Fy2));
        }
        if (r < st.nrows) {
          const R4<float> G = Gs[r * TILE_X];
          const R4<float> E = Es[r * 4];
          const T Ere(E.x, E.y), Eim(E.z, E.w);
          Fx = fma(T(G.x), Ere, fma(T(-G.y), Eim, Fx));
          Fy = fma(T(G.z), Ere, fma(T(-G.w), Eim, Fy));
        }
        Fx += Fx2;
        Fy += Fy2;
      } else {
        // the same sums in the same order as the staged path (even rows into Fx, Fy, odd rows
        // into Fx2, Fy2), so the two give the same bits
        T Fx2(0.0f), Fy2(0.0f);
        for (int r = 0; r < st.nrows; ++r) {
          const R4<float> G = st.G_cur[(long long)r * g.nx + x];
          // yA = y0 + 2 ly (even): yA and yB = yA + 1 share one entry of the phase table
          const R4<float> E = *reinterpret_cast<const R4<float> *>(reinterpret_cast<const float *>(st.EY) +
                                                                   (long long)r * 2 * st.eyp + ey_index(yA));
          const T Ere(E.x, E.y), Eim(E.z, E.w);
          if (r & 1) {
            Fx2 = fma(T(G.x), Ere, fma(T(-G.y), Eim, Fx2));
            Fy2 = fma(T(G.z), Ere, fma(T(-G.w), Eim, Fy2));
          } else {
            Fx = fma(T(G.x), Ere, fma(T(-G.y), Eim, Fx));
            Fy = fma(T(G.z), Ere, fma(T(-G.w), Eim, Fy));
          }
        }
        Fx += Fx2;
        Fy += Fy2;
      }
    }
    if (macro_out) {  // the cells' Landau solutions, forces and streamed h, kept for the reverse sweep
      const long long nc = (long long)g.nx * g.ny;
      if (flA) {
        const long long c = (long long)yA * g.nx + x;
        macro_out[c] = m.eps_m1.v.x;
        macro_out[nc + c] = m.vx.v.x;
        macro_out[2 * nc + c] = m.vy.v.x;
        macro_out[3 * nc + c] = Fx.v.x;
        macro_out[4 * nc + c] = Fy.v.x;
#pragma unroll
        for (int q = 0; q < Q; ++q) macro_out[(5 + q) * nc + c] = h[q].v.x;
      }
      if (flB) {
        const long long c = (long long)yB * g.nx + x;
        macro_out[c] = m.eps_m1.v.y;
        macro_out[nc + c] = m.vx.v.y;
        macro_out[2 * nc + c] = m.vy.v.y;
        macro_out[3 * nc + c] = Fx.v.y;
        macro_out[4 * nc + c] = Fy.v.y;
#pragma unroll
        for (int q = 0; q < Q; ++q) macro_out[(5 + q) * nc + c] = h[q].v.y;
      }
    }
    // the output in the stored scale (FP16: 2^8 h)
    constexpr float up = HScale<S>::up;
    const Coll<T> cf = coll_coeffs<T, VS, FORCE>(M, m, T(p.omega0 * up), T(p.fpref * up), Fx, Fy, T(up));
    collide_all<T, VS, FORCE>(cf, h, hn);
  }
  // a lane without fluid stores the rest state (0)
  if (!both) {
#pragma unroll
    for (int q = 0; q < Q; ++q) hn[q] = T(flA ? hn[q].v.x : 0.0f, flB ? hn[q].v.y : 0.0f);
  }
  // round once to the storage type (the ghost images below repeat the same values)
  S sA[Q], sB[Q];
  {
    const bool sr = sizeof(S) == 2 && p.stochastic;
    uint32_t rA = sr ? cell_hash(x, yA + p.y_off, p.step, p.round_key) : 0u;
    uint32_t rB = sr ? cell_hash(x, yB + p.y_off, p.step, p.round_key) : 0u;
    if constexpr (std::is_same<S, __half>::value) {
      if (sr) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          rA = next_bits(rA);
          rB = next_bits(rB);
          const uint32_t d = round_pair_f16_sr(hn[q].v.x, hn[q].v.y, rA, rB);
          sA[q] = __ushort_as_half((unsigned short)(d & 0xffffu));
          sB[q] = __ushort_as_half((unsigned short)(d >> 16));
        }
      } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const uint32_t d = round_pair_f16_rn(hn[q].v.x, hn[q].v.y);
          sA[q] = __ushort_as_half((unsigned short)(d & 0xffffu));
          sB[q] = __ushort_as_half((unsigned short)(d >> 16));
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        rA = next_bits(rA);
        rB = next_bits(rB);
        sA[q] = store_round<S>(hn[q].v.x, sr, rA);
        sB[q] = store_round<S>(hn[q].v.y, sr, rB);
      }
    }
  }
  {  // coalesced stores straight from registers (one 128-byte line per warp and plane)
    S *oA = fout + (long long)(yA + 1) * g.pitch + x + TL::XOFF;
    S *oB = oA + g.pitch;
    if (inA) {
#pragma unroll
      for (int q = 0; q < Q; ++q) oA[q * g.plane] = sA[q];
    }
    if (inB) {
#pragma unroll
      for (int q = 0; q < Q; ++q) oB[q * g.plane] = sB[q];
    }
  }
  // ghost copies of the periodic neighbours (boundary cells only)
#pragma unroll
  for (int lane = 0; lane < 2; ++lane) {
    const int y = lane ? yB : yA;
    if (!(lane ? inB : inA)) continue;
    const int gxv = ghost_col(x, g.nx, g.walls);
    const int gyv = ghost_row(y, g.ny, g.walls);
    if (gxv == INT_MIN && gyv == INT_MIN) continue;
    const int px[3] = {gxv, x, gxv}, py[3] = {y, gyv, gyv};
    for (int a = 0; a < 3; ++a) {
      if (px[a] == INT_MIN || py[a] == INT_MIN) continue;
      S *o = fout + (long long)(py[a] + 1) * g.pitch + px[a] + TL::XOFF;
#pragma unroll
      for (int q = 0; q < Q; ++q) o[q * g.plane] = lane ? sB[q] : sA[q];
    }
  }
}

// ---------------------------------------------------------------------------
// The fused step (procedure items 2-5 of Sec. "The Standard/Classical LBM", with the
// driving term of Sec. "The Driving Term").  Persistent CTAs walk the 32 x 8 tiles of
// the lattice.  Per tile, one 3-D TMA copy stages all Q planes of the tile plus a
// one-cell halo (ghost rows/columns carry the periodic wrap) into shared memory, with
// the tile's stirring rows; NST stages rotate on mbarriers (NST = 2: the next tile is
// in flight while this one is computed; NST = 1: more CTAs per SM hide the copy
// instead).  Each thread pull-streams its cell(s) from shared memory (bilinear
// weights, bounce-back substitution from the mask), takes the moments, Landau-matches,
// relaxes, adds the force and stores the Q results with coalesced stores, refreshing
// the ghost copies of boundary cells.
// ---------------------------------------------------------------------------
template <typename S, int VS, bool MASK, bool FORCE, int CPT, int NST, bool STORE>
__global__ void __launch_bounds__(NTHREADS / CPT)
step_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tG,
            const __grid_constant__ CUtensorMap tEY, S *__restrict__ fout,
            const Geometry<typename RealOf<S>::type> g, const Physics<typename RealOf<S>::type> p,
            const Stir<typename RealOf<S>::type> st, int prep_bytes, int srows_in, int *__restrict__ tile_ctr,
            unsigned seq, unsigned *__restrict__ err, typename RealOf<S>::type *__restrict__ macro_out) {
  using R = typename RealOf<S>::type;
  using TL = Tile<S, VS>;
  constexpr int NT = NTHREADS / CPT;
  const int wid = blockIdx.x, nworkers = gridDim.x;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // every TMA box lands on a 128-byte boundary of this aligned base
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  // stirring rows staged with the tile (srows_in > 0) or read from global memory (L2)
  const bool staged = FORCE && srows_in > 0;
  const int srows = staged ? srows_in : 0;
  const int stage_stride = TL::stage(srows), ey_off = TL::IN_STRIDE + TL::g_bytes(srows);
  // barriers: one per stage, then one for the mode data; then the tile of each stage
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + NST * stage_stride);
  int *tile_of = reinterpret_cast<int *>(smem + NST * stage_stride + 32);
  int *tile_xy = tile_of + NST;  // the stage's tile column | row << 16, set with tile_of

  const int tid = threadIdx.x;
  const int ntx = (g.nx + TILE_X - 1) / TILE_X, nty = (g.ny + TILE_Y - 1) / TILE_Y;
  const int ntiles = ntx * nty;
  const float rcp_ntx = 1.0f / (float)ntx;
  const uint32_t stage_bytes = TL::IN_BYTES + srows * (TL::G_ROW + TL::EY_ROW);
  // The mode data of step n+1 (coefficients, k_x, row ranges), copied on its own barrier
  // when it fits in the `prep` area past the barriers.
  constexpr int RB = (int)sizeof(R);
  const int cb = mode_coef_bytes(st.nmodes, RB), kb = mode_kx_bytes(st.nmodes), rb_ = mode_rows_bytes(st.nrows);
  const bool prep_copy = FORCE && st.nrows > 0 && cb + kb + rb_ <= prep_bytes;
  unsigned char *prep = smem + NST * stage_stride + 64;
  // Tiles are handed out by a counter of this launch (launches alternate between two; the
  // first CTA clears the other one for the next launch).  Every tile is computed the same
  // way by whichever CTA takes it, so the results do not depend on the order.
  int *ctr = tile_ctr + (seq & 1u);

  if (tid == 0) {
    for (int s = 0; s <= NST; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  // A launch chained to the previous step (programmatic dependent launch) may start while
  // that step's grid drains: the state, the stirring tables, the mode data and the tile
  // counters it wrote are touched only after it has completed and its writes are visible.
  griddep_wait();
  if (tid == 0 && wid == 0) tile_ctr[(seq + 1u) & 1u] = 0;
  __syncthreads();
  // thread 0: stage s takes tile t (or, with t past the end, only completes its barrier:
  // this CTA takes no further tile, and the next step's grid, when chained, may be
  // scheduled once every CTA has come this far)
  auto fill = [&](int s, int t) {
    uint64_t *b = &bar[s];
    tile_of[s] = t < ntiles ? t : -1;
    if (t >= ntiles) {
      mbar_arrive(b);
      griddep_launch_dependents();
      return;
    }
    // row = t / ntx, column = t mod ntx: the float quotient corrected exactly (t < 2^24)
    int row = (int)((float)t * rcp_ntx), col = t - row * ntx;
    while (col < 0) { --row; col += ntx; }
    while (col >= ntx) { ++row; col -= ntx; }
    tile_xy[s] = col | (row << 16);
    const int x0 = col * TILE_X, y0 = row * TILE_Y;
    unsigned char *st0 = smem + s * stage_stride;
    mbar_expect_tx(b, stage_bytes);
    tma_load_3d(st0, &tin, b, x0 + TL::XOFF - TL::V, y0, 0);
    if (staged) {
      tma_load_2d(st0 + TL::IN_STRIDE, &tG, b, 4 * x0, 0);
      tma_load_2d(st0 + ey_off, &tEY, b, 2 * y0, 0);
    }
  };
  int pending = 0;  // thread 0: the tile the next refill will stage (fetched one tile ahead)
  if (tid == 0) {
    if (prep_copy) {
      mbar_expect_tx(&bar[NST], cb + kb + rb_);
      bulk_load(prep, st.coef_next, cb, &bar[NST]);
      bulk_load(prep + cb, st.mode_kx, kb, &bar[NST]);
      bulk_load(prep + cb + kb, st.row_start, rb_, &bar[NST]);
    }
    for (int s = 0; s < NST; ++s) fill(s, atomicAdd(ctr, 1));
    pending = atomicAdd(ctr, 1);
  }

  // While the first tiles are in flight: for the CTAs of highest index, one Philox draw
  // of step n+2 (pure arithmetic; the multipliers are read only when they differ from 1),
  // and this CTA's share of the table of step n+1 (entry e to CTA e mod nworkers).
  if (FORCE && st.nrows && tid == 32) stir_draws_part<R>(st, nworkers - 1 - wid, nworkers);
  bool alive = true;
  if (FORCE && st.nrows) {
    if (prep_copy) {
      const bool ok = mbar_wait_bounded(&bar[NST], 0, WAIT_CYCLES);
      if (__syncthreads_or(!ok)) alive = false;
      if (alive) {
        const R4<R> *cs = reinterpret_cast<const R4<R> *>(prep);
        const int *ks = reinterpret_cast<const int *>(prep + cb), *rs = reinterpret_cast<const int *>(prep + cb + kb);
        stir_table_staged<R>(st, wid, nworkers, tid, NT, g.nx, cs, ks, rs);
      }
    } else {
      stir_table_part<R>(st, wid, nworkers, tid, NT, g.nx, nullptr, 0);
    }
  }

  // Every thread waits for the staged tile (bounded); the vote in the barrier makes the
  // whole CTA wind down together if a copy never lands.
  if (alive) {
    const bool ok = mbar_wait_bounded(&bar[0], 0, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) alive = false;
  }
  for (int k = 0; alive; ++k) {
    const int s = k % NST;
    const int t = tile_of[s];
    if (t < 0) break;
    const int xy = tile_xy[s];
    tile_cells<S, VS, MASK, FORCE, CPT>(smem + s * stage_stride, ey_off, fout, (xy & 0xffff) * TILE_X,
                                        (xy >> 16) * TILE_Y, tid, g, g, p, st, staged, err,
                                        STORE ? macro_out : static_cast<R *>(nullptr));
    if (NST == 1) {  // the only stage is free once every thread is done with it
      __syncthreads();
      if (tid == 0) {
        fill(0, pending);
        pending = atomicAdd(ctr, 1);
      }
    }
    // the next stage's barrier completes with its tile, or at once when it has none
    const int sn = (k + 1) % NST;
    const bool ok = mbar_wait_bounded(&bar[sn], ((k + 1) / NST) & 1, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) {  // (NST = 2: also the barrier after which stage s is free)
      alive = false;
      break;
    }
    if (NST >= 2 && tid == 0) {
      fill(s, pending);
      pending = atomicAdd(ctr, 1);
    }
  }
  if (!alive && tid == 0) {
    // a staged copy did not land in time: latch the error and wait (bounded) once more
    // for this CTA's copies still in flight before returning
    atomicOr(err, ERR_TIMEOUT);
    for (int s2 = 0; s2 <= NST; ++s2) mbar_wait_bounded(&bar[s2], 0, WAIT_CYCLES);
  }
}

// ---------------------------------------------------------------------------
// The batched step: one persistent launch advances every lattice of a batch (an
// ensemble of stirred realisations or impurity samples, uneven sizes) by one step.
// The tiles of all members form one list (member m owns tiles tile0[m] .. tile0[m+1]);
// CTAs walk it exactly as the single-lattice kernel walks one lattice (tiles handed out
// by a counter, cleared between launches by the kernel that advances the step), and take
// each tile's member (searched forward from the CTA's previous tile's member), buffers and
// TMA descriptors from the member table; the thread that stages a tile resolves it once
// and leaves what the tile needs in shared memory beside the stage.
// The per-member step is step0 + *bstep, so a captured CUDA graph of launches can
// replay with the counter advanced by a one-thread kernel between launches.  All members
// share the velocity set, storage type, dt/a, eta/s, eps0, the force shell and the
// rounding mode; they differ in size, walls, solids, seeds and initial fields.
// ---------------------------------------------------------------------------
struct BatchDims {
  int nx, ny, pitch, walls;
  long long plane;
  const uint16_t *nbmask;
};

// What the cells of a staged tile need of its member (written by the staging thread).
struct alignas(16) TileInfo {
  BatchDims dims;
  void *fout;          // the buffer this step writes
  unsigned *err;
  long long n;         // the member's step index
  int x0, y0, m;
  unsigned round_key;
};

__device__ __forceinline__ int find_member(const int *prefix, int n, int t) {
  int lo = 0, hi = n;  // prefix[lo] <= t < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

template <typename R> __device__ __forceinline__ Stir<R> member_stir(const MemberDesc &d, long long n) {
  Stir<R> s;
  s.nrows = d.nrows; s.nmodes = d.nmodes; s.eyp = d.eyp;
  s.G_cur = (const R4<R> *)d.G[n & 1];
  s.EY = (const R2<R> *)d.EY;
  s.G_next = (R4<R> *)d.G[(n + 1) & 1];
  s.coef_next = (const R4<R> *)d.coef[(n + 1) & 1];
  s.coef_new = (R4<R> *)d.coef[n & 1];
  s.mode_kx = d.mode_kx; s.row_start = d.row_start;
  s.seed = d.seed; s.step_new = n + 2; s.amp = 0.0; s.mode_scale = nullptr;
  return s;
}

template <typename S, int VS, bool MASK, bool FORCE, int CPT, int NST>
__global__ void __launch_bounds__(NTHREADS / CPT, CPT == 2 ? 4 : 1)  // two-cell paths: 4 CTAs/SM
batch_step_kernel(const BatchTables bt, const Geometry<typename RealOf<S>::type> wts,
                  const Physics<typename RealOf<S>::type> p0, const int srows_in, const double amp,
                  const long long *__restrict__ bstep_ptr) {
  using R = typename RealOf<S>::type;
  using TL = Tile<S, VS>;
  constexpr int NT = NTHREADS / CPT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const bool staged = FORCE && srows_in > 0;
  const int srows = staged ? srows_in : 0;
  const int stage_stride = TL::stage(srows), ey_off = TL::IN_STRIDE + TL::g_bytes(srows);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + NST * stage_stride);
  TileInfo *info = reinterpret_cast<TileInfo *>(smem + NST * stage_stride + 64);
  const uint32_t stage_bytes = TL::IN_BYTES + srows * (TL::G_ROW + TL::EY_ROW);
  const long long bstep = *bstep_ptr;

  const int tid = threadIdx.x, wid = blockIdx.x, nworkers = gridDim.x;
  const int ntiles = bt.tile0[bt.n];
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // thread 0: stage s takes tile t of the list (handed out by the launch's counter, so a
  // CTA that runs ahead takes more tiles), or, with t past the end, only completes its
  // barrier; the tile's member is resolved here, once, into the stage's TileInfo.  A CTA's
  // tiles only increase, so the member search starts at the previous tile's member.
  int m_last = 0;
  auto fill = [&](int s, int t) {
    TileInfo &ti = info[s];
    uint64_t *b = &bar[s];
    if (t >= ntiles) {
      ti.m = -1;
      mbar_arrive(b);
      return;
    }
    int m = m_last;
    while (bt.tile0[m + 1] <= t) ++m;  // tile0[n] = ntiles > t ends the search
    m_last = m;
    const MemberDesc &d = bt.mem[m];
    const int lt = t - bt.tile0[m];
    // row = lt / ntx, column = lt mod ntx: the float quotient is within a unit or two of
    // the exact one (lt < 2^24), then corrected exactly
    int row = (int)((float)lt * d.rcp_ntx), col = lt - row * d.ntx;
    while (col < 0) { --row; col += d.ntx; }
    while (col >= d.ntx) { ++row; col -= d.ntx; }
    const int x0 = col * TILE_X, y0 = row * TILE_Y;
    const long long n = d.step0 + bstep;
    const int cur = (d.cur0 + (int)(bstep & 1)) & 1;
    ti.dims = BatchDims{d.nx, d.ny, d.pitch, d.walls, d.plane, d.nbmask};
    ti.fout = d.f[cur ^ 1];
    ti.err = d.err;
    ti.n = n;
    ti.x0 = x0;
    ti.y0 = y0;
    ti.m = m;
    ti.round_key = d.round_key;
    unsigned char *st0 = smem + s * stage_stride;
    mbar_expect_tx(b, stage_bytes);
    tma_load_3d(st0, &d.tin[cur], b, x0 + TL::XOFF - TL::V, y0, 0);
    if (staged) {
      tma_load_2d(st0 + TL::IN_STRIDE, &d.tG[n & 1], b, 4 * x0, 0);
      tma_load_2d(st0 + ey_off, &d.tEY, b, 2 * y0, 0);
    }
  };
  int pending = 0;  // thread 0: the tile the next refill will stage (fetched one tile ahead)
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) fill(s, atomicAdd(bt.tile_ctr, 1));
    pending = atomicAdd(bt.tile_ctr, 1);
  }
  bool alive = true;
  {
    const bool ok = mbar_wait_bounded(&bar[0], 0, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) alive = false;
  }
  for (int k = 0; alive; ++k) {
    const int s = k % NST;
    const TileInfo ti = info[s];
    if (ti.m < 0) break;
    Physics<R> p = p0;
    p.round_key = ti.round_key;
    p.step = (unsigned)(ti.n & 0xffffffffll);
    // staged stirring rows need only their count (the shell is shared by all members)
    Stir<R> st{};
    if (FORCE && staged) st.nrows = srows;
    else if (FORCE) st = member_stir<R>(bt.mem[ti.m], ti.n);
    tile_cells<S, VS, MASK, FORCE, CPT>(smem + s * stage_stride, ey_off, (S *)ti.fout, ti.x0, ti.y0, tid, ti.dims,
                                        wts, p, st, staged, ti.err, static_cast<R *>(nullptr));
    if (NST == 1) {  // the only stage is free once every thread is done with it
      __syncthreads();
      if (tid == 0) {
        fill(0, pending);
        pending = atomicAdd(bt.tile_ctr, 1);
      }
    }
    // the next stage's barrier completes with its tile, or at once when it has none
    const int sn = (k + 1) % NST;
    const bool ok = mbar_wait_bounded(&bar[sn], ((k + 1) / NST) & 1, WAIT_CYCLES);
    if (__syncthreads_or(!ok)) {  // (NST = 2: also the barrier after which stage s is free)
      alive = false;
      break;
    }
    if (NST >= 2 && tid == 0) {
      fill(s, pending);
      pending = atomicAdd(bt.tile_ctr, 1);
    }
  }
  if (!alive && tid == 0) {
    atomicOr(bt.mem[0].err, ERR_TIMEOUT);
    for (int s2 = 0; s2 < NST; ++s2) mbar_wait_bounded(&bar[s2], 0, WAIT_CYCLES);
  }
  if (!alive) return;  // copies may still be in flight: stage 0 is not free
  // The stirring work of the following steps, after the tiles: table entries of step n+1,
  // then the draws of step n+2, of every member.  Each CTA takes a contiguous range of the
  // entries (members in order, entry = row * nx + x) and builds it member by member, the
  // member's mode data (coefficients of step n+1, k_x, row ranges) first copied into the
  // free stage 0; consecutive threads take consecutive entries.
  if (FORCE && srows_in >= 0 && bt.mem[0].nrows) {
    const long long entries = bt.entry0[bt.n];
    const long long per = (entries + nworkers - 1) / nworkers;
    long long e0 = (long long)wid * per;
    const long long e1 = e0 + per < entries ? e0 + per : entries;
    while (e0 < e1) {
      int m = 0, hi = bt.n;  // entry0[m] <= e0 < entry0[hi]
      while (hi - m > 1) { const int mid = (m + hi) >> 1; if (bt.entry0[mid] <= e0) m = mid; else hi = mid; }
      const MemberDesc &d = bt.mem[m];
      const long long mlo = bt.entry0[m], mend = bt.entry0[m + 1] < e1 ? bt.entry0[m + 1] : e1;
      const Stir<R> st = member_stir<R>(d, d.step0 + bstep);
      const int need = st.nmodes * (int)(sizeof(R4<R>) + sizeof(int)) + (st.nrows + 1) * (int)sizeof(int);
      const R4<R> *coef = st.coef_next;
      const int *kx = st.mode_kx, *rs = st.row_start;
      if (need <= (int)TL::IN_STRIDE) {
        R4<R> *c2 = reinterpret_cast<R4<R> *>(smem);
        int *k2 = reinterpret_cast<int *>(c2 + st.nmodes);
        int *r2 = k2 + st.nmodes;
        for (int i = tid; i < st.nmodes; i += NT) { c2[i] = coef[i]; k2[i] = kx[i]; }
        for (int i = tid; i <= st.nrows; i += NT) r2[i] = rs[i];
        __syncthreads();
        coef = c2; kx = k2; rs = r2;
      }
      const int nx = d.nx;
      for (long long e = e0 + tid; e < mend; e += NT) {
        const int le = (int)(e - mlo);  // < nrows * nx
        st.G_next[le] = stir_row_entry<R>(coef, kx, rs, le / nx, le % nx, nx);
      }
      __syncthreads();  // the staged mode data is replaced by the next member's
      e0 = mend;
    }
    const int draws = bt.draw0[bt.n];
    const int dper = (draws + nworkers - 1) / nworkers;
    const int d1 = (wid + 1) * dper < draws ? (wid + 1) * dper : draws;
    for (int e = wid * dper + tid; e < d1; e += NT) {
      const int m = find_member(bt.draw0, bt.n, e);
      const MemberDesc &d = bt.mem[m];
      Stir<R> st = member_stir<R>(d, d.step0 + bstep);
      st.amp = amp;
      stir_draws_part<R>(st, e - bt.draw0[m], st.nmodes);
    }
  }
}

// ---------------------------------------------------------------------------
// Moments of the current state f_n = stream(f*_n) (procedure item 3) straight from
// global memory (ghost-padded planes): eps, u^x, u^y per cell and per-block FP64
// partial sums of T^00, T^0x, T^0y, 1/2 |v|^2.  Landau runs in FP64 here.
// ---------------------------------------------------------------------------
template <typename S, typename R, int VS, bool MASK>
__device__ __forceinline__ void pull_global(const S *__restrict__ fin, const Geometry<R> &g, int x, int y,
                                            unsigned nb, R h[VSet<VS>::Q]) {
  constexpr int Q = VSet<VS>::Q;
  const long long o = (long long)(y + 1) * g.pitch + x + PadLayout<S>::XOFF;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const S *pl = fin + q * g.plane + o;
    const int sx = sgnx<VS>(q), sy = sgny<VS>(q);
    R acc = g.beta[q][0] * load_h<S, R>(pl);
    const R own = load_h<S, R>(fin + VSet<VS>::opp(q) * g.plane + o);
    if (sx != 0) acc += g.beta[q][1] * ((MASK && ((nb >> (4 - sx)) & 1u)) ? own : load_h<S, R>(pl - sx));
    if (sy != 0) acc += g.beta[q][2] * ((MASK && ((nb >> (4 - 3 * sy)) & 1u)) ? own : load_h<S, R>(pl - (long long)sy * g.pitch));
    if (sx != 0 && sy != 0)
      acc += g.beta[q][3] * ((MASK && ((nb >> (4 - 3 * sy - sx)) & 1u)) ? own : load_h<S, R>(pl - (long long)sy * g.pitch - sx));
    h[q] = acc;
  }
}

template <typename S, int VS, bool MASK>
__global__ void __launch_bounds__(256)
moments_kernel(const S *__restrict__ fin, const Geometry<typename RealOf<S>::type> g, double eps0, float vmax2,
               double *__restrict__ eps, double *__restrict__ ux, double *__restrict__ uy,
               double *__restrict__ partials, unsigned *__restrict__ err) {
  using R = typename RealOf<S>::type;
  constexpr int Q = VSet<VS>::Q;
  constexpr bool F64 = sizeof(R) == 8;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  // Per-cell terms of the block totals: T^00, T^0x, T^0y, 1/2 |v|^2.  FP64 storage sums
  // them in FP64.  The other storage types (FP32 state) match and sum in FP32, as the step
  // kernel does (GB300's FP64 rate is 1/64 of FP32): the FP32 terms are the deviations
  // e, m_x, m_y (order u), summed per warp, and the warps' sums are added in FP64 to the
  // exact count of fluid cells (T^00 = eps0 (1 + e)).
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float accf[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  int fluid = 0;
  if (x < g.nx && y < g.ny) {
    const long long c = (long long)y * g.nx + x;
    unsigned nb = MASK ? g.nbmask[c] : 0u;
    if (MASK && (nb & 16u)) {
      eps[c] = 0.0; ux[c] = 0.0; uy[c] = 0.0;
    } else {
      R h[Q];
      pull_global<S, R, VS, MASK>(fin, g, x, y, nb, h);
      if constexpr (F64) {
        const Mom<double> M = moments_of<double, R, VS, false>(h);
        const Macro<double> m = macro_from<double, VS>(M, 40, 1e-12);
        if (!m.ok) atomicOr(err, (1.0 + m.eps_m1 > 0.0 && isfinite(m.eps_m1)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
        eps[c] = eps0 * (1.0 + m.eps_m1);
        ux[c] = m.ux;
        uy[c] = m.uy;
        acc[0] = eps0 * (1.0 + M.e);
        acc[1] = eps0 * M.mx;
        acc[2] = eps0 * M.my;
        acc[3] = 0.5 * (m.vx * m.vx + m.vy * m.vy);
      } else {
        // Landau in FP32, re-solved in FP64 where it has not converged or |v| > vmax
        const Mom<float> M = moments_of<float, float, VS, false>(h);
        const Macro<float> m = cell_macro<float, VS>(h, M, vmax2);
        if (!m.ok) atomicOr(err, (1.0f + m.eps_m1 > 0.0f && isfinite(m.eps_m1)) ? ERR_UNPHYSICAL : ERR_UNSTABLE);
        eps[c] = eps0 * (1.0 + (double)m.eps_m1);
        ux[c] = m.ux;
        uy[c] = m.uy;
        accf[0] = M.e;
        accf[1] = M.mx;
        accf[2] = M.my;
        accf[3] = 0.5f * (m.vx * m.vx + m.vy * m.vy);
        fluid = 1;
      }
    }
  }
  __shared__ double red[4][32];
  __shared__ int cnt[32];
  const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
  const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if constexpr (F64) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double v = acc[k];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[k][warp] = v;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float v = accf[k];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[k][warp] = (double)v;
    }
    const int nf = __popc(__ballot_sync(0xffffffffu, fluid));
    if (lane == 0) cnt[warp] = nf;
  }
  __syncthreads();
  const int nwarps = (blockDim.x * blockDim.y + 31) / 32;
  if (warp == 0) {
    double tot[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double v = lane < nwarps ? red[k][lane] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      tot[k] = v;
    }
    if (!F64) {
      int nf = lane < nwarps ? cnt[lane] : 0;
      for (int off = 16; off > 0; off >>= 1) nf += __shfl_down_sync(0xffffffffu, nf, off);
      tot[0] = eps0 * ((double)nf + tot[0]);
      tot[1] *= eps0;
      tot[2] *= eps0;
    }
    if (lane == 0)
      for (int k = 0; k < 4; ++k) partials[(long long)(blockIdx.y * gridDim.x + blockIdx.x) * 4 + k] = tot[k];
  }
}

// ---------------------------------------------------------------------------
// Initial state f*_0 = f_eq(eps, u) (procedure item 1); NULL fields mean eps0 at rest.
// Writes the interior; ghost copies come from fill_ghosts.
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
  const long long o = (long long)(y + 1) * g.pitch + x + PadLayout<S>::XOFF;
#pragma unroll
  for (int q = 0; q < V::Q; ++q) {
    const double uv = ax * V::vx(q) + ay * V::vy(q);
    const double heq = (e - 1.0) + V::CA * e * u0 * uv + V::CB * e * uv * uv - V::CC * e * u2;
    fout[q * g.plane + o] = store_h<S, typename RealOf<S>::type>((typename RealOf<S>::type)(solid ? 0.0 : heq));
  }
}

// Ghost columns (x = -1, nx) and, for periodic y, ghost rows (y = -1, ny) and corners:
// copies of the wrapped interior.  With walls the ghost rows stay zero.
template <typename S, int VS>
__global__ void fill_ghosts_kernel(S *__restrict__ f, const Geometry<typename RealOf<S>::type> g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  const int nper = 2 * (g.ny + 2) + 2 * g.nx;
  if (i >= nper) return;
  int gx, gy;  // ghost coordinate in cell units (-1 .. nx, -1 .. ny)
  if (i < 2 * (g.ny + 2)) { gx = (i & 1) ? g.nx : -1; gy = i / 2 - 1; }
  else { const int j = i - 2 * (g.ny + 2); gx = j / 2; gy = (j & 1) ? g.ny : -1; }
  S *pl = f + q * g.plane;
  const long long dst = (long long)(gy + 1) * g.pitch + gx + PadLayout<S>::XOFF;
  const bool yghost = gy < 0 || gy >= g.ny;
  if (yghost && (g.walls & STRIP_Y)) return;  // a strip's ghost rows come from the halo exchange
  if (yghost && (g.walls & WALLS_Y)) { pl[dst] = store_h<S, typename RealOf<S>::type>(0); return; }
  const int sx = (gx + g.nx) % g.nx, sy = (gy + g.ny) % g.ny;
  pl[dst] = pl[(long long)(sy + 1) * g.pitch + sx + PadLayout<S>::XOFF];
}

// Open channel (walls bit OPEN_X): the column left of x = 0 holds the inflow equilibrium
// (eps0, u^x = ux_in; written here once and never by the step kernel) and the column right
// of x = nx - 1 repeats that column (zero-gradient outflow; the step kernel keeps it up).
// Rows of bounce-back walls stay zero.  One thread per padded row, one grid row per plane.
template <typename S, int VS>
__global__ void open_ghosts_kernel(S *__restrict__ f, const Geometry<typename RealOf<S>::type> g, double ux_in) {
  using V = VSet<VS>;
  using R = typename RealOf<S>::type;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;  // padded row 0 .. ny + 1
  const int q = blockIdx.y;
  if (row >= g.ny + 2) return;
  S *pl = f + q * g.plane + (long long)row * g.pitch + PadLayout<S>::XOFF;
  pl[g.nx] = pl[g.nx - 1];
  const bool wall_row = (g.walls & WALLS_Y) && (row == 0 || row == g.ny + 1);
  const double u0 = sqrt(1.0 + ux_in * ux_in), uv = ux_in * V::vx(q);
  const double heq = V::CA * u0 * uv + V::CB * uv * uv - V::CC * ux_in * ux_in;  // eps / eps0 = 1
  pl[-1] = store_h<S, R>((R)(wall_row ? 0.0 : heq));
}

// Stirring pipeline start at step n: coefficients of steps n and n+1, table of step n.
template <typename R>
__global__ void stir_draw_kernel(R4<R> *coef_a, R4<R> *coef_b, int nmodes, unsigned long long seed,
                                 long long n, double amp, const double *__restrict__ scale) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * nmodes) return;
  const int m = t % nmodes;
  if (scale) amp *= scale[m];
  // same arithmetic as the draws a step launch makes for later steps
  if constexpr (sizeof(R) == 8) {
    double c[4];
    stir_draw(seed, n + t / nmodes, m, amp, c);
    (t < nmodes ? coef_a : coef_b)[m] = R4<R>{(R)c[0], (R)c[1], (R)c[2], (R)c[3]};
  } else {
    float c[4];
    stir_draw_f32(seed, n + t / nmodes, m, (float)amp, c);
    (t < nmodes ? coef_a : coef_b)[m] = R4<R>{c[0], c[1], c[2], c[3]};
  }
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
// beta2, the pull weights of the paired kernels, carries 1 / HScale<S>::up: those kernels
// convert the stored values without the scale.
template <typename S> static Geometry<typename RealOf<S>::type> to_geom(const HostGeom &h) {
  using R = typename RealOf<S>::type;
  Geometry<R> g;
  g.nx = h.nx; g.ny = h.ny; g.pitch = h.pitch; g.plane = h.plane; g.walls = h.walls; g.nbmask = h.nbmask;
  for (int q = 0; q < 17; ++q)
    for (int k = 0; k < 4; ++k) {
      g.beta[q][k] = (R)h.beta[q][k];
      const float b = (float)h.beta[q][k] * HScale<S>::down;
      g.beta2[q][k] = make_float2(b, b);
    }
  return g;
}

template <typename R> static Stir<R> to_stir(const HostStir &h) {
  Stir<R> s;
  s.nrows = h.nrows; s.nmodes = h.nmodes;
  s.G_cur = (const R4<R> *)h.G_cur; s.EY = (const R2<R> *)h.EY; s.G_next = (R4<R> *)h.G_next;
  s.coef_next = (const R4<R> *)h.coef_next; s.coef_new = (R4<R> *)h.coef_new;
  s.mode_kx = h.mode_kx; s.row_start = h.row_start; s.eyp = h.eyp;
  s.seed = h.seed; s.step_new = h.step_new; s.amp = h.amp; s.mode_scale = h.mode_scale;
  return s;
}

// STORE: the variant that also keeps each fluid cell's Landau solution, force and streamed
// deviations h (5 + Q planes of nx * ny values; the gradient's recomputation); the regular
// kernel is compiled without that store.
template <typename S, int VS, bool MASK, bool FORCE, int NST, bool STORE>
static cudaError_t launch_step_k(const CUtensorMap &tin, const CUtensorMap &tG, const CUtensorMap &tEY, void *fout,
                                 const Geometry<typename RealOf<S>::type> &g, const Physics<typename RealOf<S>::type> &p,
                                 const Stir<typename RealOf<S>::type> &s, unsigned *err, int grid_limit,
                                 int stir_rows, int *tile_ctr, unsigned seq, bool chained, void *macro_out,
                                 cudaStream_t stream) {
  using TL = Tile<S, VS>;
  using R = typename RealOf<S>::type;
  constexpr int CPT = sizeof(S) == 8 ? 1 : 2;
  constexpr int NT = NTHREADS / CPT;
  auto kern = step_kernel<S, VS, MASK, FORCE, CPT, NST, STORE>;
  const int srows = (FORCE && s.nrows > 0 && s.nrows <= TL::MAX_SROWS && stir_rows != 2) ? s.nrows : 0;
  // room to stage the stirring modes of the next step (coefficients, k_x, row ranges)
  const int prep_bytes =
      (FORCE && s.nrows && s.nmodes <= 1024)
          ? (mode_coef_bytes(s.nmodes, (int)sizeof(typename RealOf<S>::type)) + mode_kx_bytes(s.nmodes) +
             mode_rows_bytes(s.nrows) + 127) / 128 * 128
          : 0;
  const int smem = TL::smem(NST, srows) + prep_bytes;
  static int configured_dev = -1, configured_smem = -1, max_blocks = 0, sms = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev != dev || configured_smem != smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_blocks, kern, NT, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    configured_dev = dev;
    configured_smem = smem;
  }
  const int ntiles = ((g.nx + TILE_X - 1) / TILE_X) * ((g.ny + TILE_Y - 1) / TILE_Y);
  int workers = max_blocks * sms;
  if (grid_limit > 0 && grid_limit < workers) workers = grid_limit;
  if (workers > ntiles) workers = ntiles;
  if (workers < 1) workers = 1;
  if (chained) {
    // a step right after the previous one on the same stream: programmatic dependent
    // launch lets its CTAs be scheduled while that step's last tiles finish
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(workers);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, tin, tG, tEY, (S *)fout, g, p, s, prep_bytes, srows, tile_ctr, seq, err,
                              static_cast<R *>(macro_out));
  }
  kern<<<workers, NT, smem, stream>>>(tin, tG, tEY, (S *)fout, g, p, s, prep_bytes, srows, tile_ctr, seq, err,
                                      static_cast<R *>(macro_out));
  return cudaGetLastError();
}

template <typename S, int VS, bool MASK, bool FORCE, int NST>
static cudaError_t launch_step_v(const CUtensorMap &tin, const CUtensorMap &tG, const CUtensorMap &tEY, void *fout,
                                 const Geometry<typename RealOf<S>::type> &g, const Physics<typename RealOf<S>::type> &p,
                                 const Stir<typename RealOf<S>::type> &s, unsigned *err, int grid_limit,
                                 int stir_rows, int *tile_ctr, unsigned seq, bool chained, void *macro_out,
                                 cudaStream_t stream) {
  if constexpr (sizeof(S) >= 4) {  // the gradient runs on FP32 and FP64 states only
    if (macro_out)
      return launch_step_k<S, VS, MASK, FORCE, NST, true>(tin, tG, tEY, fout, g, p, s, err, grid_limit, stir_rows,
                                                           tile_ctr, seq, chained, macro_out, stream);
  }
  return launch_step_k<S, VS, MASK, FORCE, NST, false>(tin, tG, tEY, fout, g, p, s, err, grid_limit, stir_rows,
                                                        tile_ctr, seq, chained, nullptr, stream);
}

template <typename S, int NST>
static cudaError_t launch_step_n(int vset, const CUtensorMap &mi, const CUtensorMap &mg, const CUtensorMap &me,
                                 void *fout, const Geometry<typename RealOf<S>::type> &g,
                                 const Physics<typename RealOf<S>::type> &p, const Stir<typename RealOf<S>::type> &s,
                                 bool mask, bool force, unsigned *err, int grid_limit, int stir_rows,
                                 int *ctr, unsigned seq, bool chained, void *macro_out, cudaStream_t stream) {
  if (vset == 3) {
    if (force) {
      if (mask) return launch_step_v<S, 3, true, true, NST>(mi, mg, me, fout, g, p, s, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
      return launch_step_v<S, 3, false, true, NST>(mi, mg, me, fout, g, p, s, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
    }
    if (mask) return launch_step_v<S, 3, true, false, NST>(mi, mg, me, fout, g, p, s, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
    return launch_step_v<S, 3, false, false, NST>(mi, mg, me, fout, g, p, s, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
  }
  if (mask) return launch_step_v<S, 2, true, false, NST>(mi, mg, me, fout, g, p, s, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
  return launch_step_v<S, 2, false, false, NST>(mi, mg, me, fout, g, p, s, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
}

template <typename S>
static cudaError_t launch_step_t(int vset, const void *tin, const void *tg, const void *tey, void *fout,
                                 const HostGeom &hg, const HostPhys &hp, const HostStir &hs, unsigned *err,
                                 int grid_limit, int stages, int stir_rows, int *ctr, unsigned seq,
                                 bool chained, void *macro_out, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<S>(hg);
  Physics<R> p;
  p.omega0 = (R)hp.omega0; p.fpref = (R)hp.fpref; p.body_x = (R)hp.body_x; p.body_y = (R)hp.body_y;
  p.vmax2 = (R)hp.vmax2;
  p.stochastic = hp.stochastic;
  p.round_key = hp.round_key;
  p.step = (unsigned)(hp.step & 0xffffffffll);
  p.y_off = hp.y_off;
  const Stir<R> s = to_stir<R>(hs);
  const CUtensorMap &mi = *(const CUtensorMap *)tin, &mg = *(const CUtensorMap *)tg, &me = *(const CUtensorMap *)tey;
  const bool mask = hg.nbmask != nullptr, force = hp.has_force != 0;
  if (stages == 1)
    return launch_step_n<S, 1>(vset, mi, mg, me, fout, g, p, s, mask, force, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
  return launch_step_n<S, 2>(vset, mi, mg, me, fout, g, p, s, mask, force, err, grid_limit, stir_rows, ctr, seq, chained, macro_out, stream);
}

template <typename S, int VS, bool MASK, bool FORCE, int NST>
static cudaError_t launch_batch_v(const BatchTables &bt, const Geometry<typename RealOf<S>::type> &w,
                                  const Physics<typename RealOf<S>::type> &p, int srows, double amp,
                                  const long long *bstep, int grid_limit, int ntiles, cudaStream_t stream) {
  using TL = Tile<S, VS>;
  constexpr int CPT = sizeof(S) == 8 ? 1 : 2;
  constexpr int NT = NTHREADS / CPT;
  auto kern = batch_step_kernel<S, VS, MASK, FORCE, CPT, NST>;
  const int smem = TL::smem(NST, FORCE ? srows : 0) + NST * (int)sizeof(TileInfo);
  static int configured_dev = -1, configured_smem = -1, max_blocks = 0, sms = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev != dev || configured_smem != smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&max_blocks, kern, NT, smem);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    configured_dev = dev;
    configured_smem = smem;
  }
  int workers = max_blocks * sms;
  if (grid_limit > 0 && grid_limit < workers) workers = grid_limit;
  if (workers > ntiles) workers = ntiles;
  if (workers < 1) workers = 1;
  kern<<<workers, NT, smem, stream>>>(bt, w, p, FORCE ? srows : 0, amp, bstep);
  return cudaGetLastError();
}

template <typename S, int NST>
static cudaError_t launch_batch_n(int vset, const BatchTables &bt, const Geometry<typename RealOf<S>::type> &w,
                                  const Physics<typename RealOf<S>::type> &p, int srows, double amp,
                                  const long long *bstep, bool mask, bool force, int grid_limit, int ntiles,
                                  cudaStream_t st) {
  if (vset == 3) {
    if (force) {
      if (mask) return launch_batch_v<S, 3, true, true, NST>(bt, w, p, srows, amp, bstep, grid_limit, ntiles, st);
      return launch_batch_v<S, 3, false, true, NST>(bt, w, p, srows, amp, bstep, grid_limit, ntiles, st);
    }
    if (mask) return launch_batch_v<S, 3, true, false, NST>(bt, w, p, srows, amp, bstep, grid_limit, ntiles, st);
    return launch_batch_v<S, 3, false, false, NST>(bt, w, p, srows, amp, bstep, grid_limit, ntiles, st);
  }
  if (mask) return launch_batch_v<S, 2, true, false, NST>(bt, w, p, srows, amp, bstep, grid_limit, ntiles, st);
  return launch_batch_v<S, 2, false, false, NST>(bt, w, p, srows, amp, bstep, grid_limit, ntiles, st);
}

template <typename S>
static cudaError_t launch_batch_t(int vset, const BatchTables &bt, const HostGeom &hw, const HostPhys &hp, int srows,
                                  double amp, const long long *bstep, bool mask, int stages, int grid_limit,
                                  int ntiles, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> w = to_geom<S>(hw);
  Physics<R> p;
  p.omega0 = (R)hp.omega0; p.fpref = (R)hp.fpref; p.body_x = (R)hp.body_x; p.body_y = (R)hp.body_y;
  p.vmax2 = (R)hp.vmax2;
  p.stochastic = hp.stochastic;
  p.round_key = 0;
  p.step = 0;
  p.y_off = 0;
  const bool force = hp.has_force != 0;
  if (stages == 1)
    return launch_batch_n<S, 1>(vset, bt, w, p, srows, amp, bstep, mask, force, grid_limit, ntiles, stream);
  return launch_batch_n<S, 2>(vset, bt, w, p, srows, amp, bstep, mask, force, grid_limit, ntiles, stream);
}

template <typename S>
static cudaError_t launch_moments_t(int vset, const void *fin, const HostGeom &hg, double eps0, double vmax2,
                                    double *eps, double *ux, double *uy, double *partials, unsigned *err,
                                    dim3 block, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<S>(hg);
  const dim3 grid((hg.nx + block.x - 1) / block.x, (hg.ny + block.y - 1) / block.y);
  const bool mask = hg.nbmask != nullptr;
  const S *a = (const S *)fin;
  if (vset == 3) {
    if (mask) moments_kernel<S, 3, true><<<grid, block, 0, stream>>>(a, g, eps0, (float)vmax2, eps, ux, uy, partials, err);
    else moments_kernel<S, 3, false><<<grid, block, 0, stream>>>(a, g, eps0, (float)vmax2, eps, ux, uy, partials, err);
  } else {
    if (mask) moments_kernel<S, 2, true><<<grid, block, 0, stream>>>(a, g, eps0, (float)vmax2, eps, ux, uy, partials, err);
    else moments_kernel<S, 2, false><<<grid, block, 0, stream>>>(a, g, eps0, (float)vmax2, eps, ux, uy, partials, err);
  }
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_ghosts_t(int vset, void *f, const HostGeom &hg, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<S>(hg);
  const int nper = 2 * (hg.ny + 2) + 2 * hg.nx;
  const dim3 grid((nper + 255) / 256, vset == 3 ? VSet<3>::Q : VSet<2>::Q);
  if (vset == 3) fill_ghosts_kernel<S, 3><<<grid, 256, 0, stream>>>((S *)f, g);
  else fill_ghosts_kernel<S, 2><<<grid, 256, 0, stream>>>((S *)f, g);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_init_t(int vset, void *fout, const HostGeom &hg, double eps0, const double *eps,
                                 const double *ux, const double *uy, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<S>(hg);
  const dim3 block(32, 8);
  const dim3 grid((hg.nx + 31) / 32, (hg.ny + 7) / 8);
  if (vset == 3) init_kernel<S, 3><<<grid, block, 0, stream>>>((S *)fout, g, eps0, eps, ux, uy);
  else init_kernel<S, 2><<<grid, block, 0, stream>>>((S *)fout, g, eps0, eps, ux, uy);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_ghosts_t<S>(vset, fout, hg, stream);
}

template <typename S>
static cudaError_t launch_open_ghosts_t(int vset, void *f, const HostGeom &hg, double ux_in, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  const Geometry<R> g = to_geom<S>(hg);
  const dim3 grid((hg.ny + 2 + 127) / 128, vset == 3 ? VSet<3>::Q : VSet<2>::Q);
  if (vset == 3) open_ghosts_kernel<S, 3><<<grid, 128, 0, stream>>>((S *)f, g, ux_in);
  else open_ghosts_kernel<S, 2><<<grid, 128, 0, stream>>>((S *)f, g, ux_in);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t launch_stir_prime_t(const HostStir &hs, void *coef_n, void *coef_n1, void *G_n, int nx,
                                       long long n, cudaStream_t stream) {
  using R = typename RealOf<S>::type;
  if (hs.nmodes == 0) return cudaSuccess;
  const Stir<R> s = to_stir<R>(hs);
  stir_draw_kernel<R><<<(2 * hs.nmodes + 127) / 128, 128, 0, stream>>>((R4<R> *)coef_n, (R4<R> *)coef_n1,
                                                                        hs.nmodes, hs.seed, n, hs.amp,
                                                                        hs.mode_scale);
  const long long entries = (long long)hs.nrows * nx;
  stir_table_kernel<R><<<(unsigned)((entries + 255) / 256), 256, 0, stream>>>(s, (R4<R> *)G_n,
                                                                             (const R4<R> *)coef_n, nx);
  return cudaGetLastError();
}

}  // namespace rlbm

#define RLBM_DEFINE_LAUNCHERS(S, SUF)                                                                    \
  namespace rlbm {                                                                                       \
  cudaError_t launch_step_##SUF(int vset, const void *tin, const void *tg, const void *tey, void *fout,     \
                                const HostGeom &g, const HostPhys &p, const HostStir &s, unsigned *err, \
                                int grid_limit, int stages, int stir_rows, int *ctr, unsigned seq,      \
                                bool chained, void *macro_out, cudaStream_t st) {                        \
    return launch_step_t<S>(vset, tin, tg, tey, fout, g, p, s, err, grid_limit, stages, stir_rows, ctr, seq, \
                            chained, macro_out, st);                                                    \
  }                                                                                                      \
  cudaError_t launch_batch_step_##SUF(int vset, const BatchTables &bt, const HostGeom &w, const HostPhys &p, \
                                      int srows, double amp, const long long *bstep, bool mask, int stages, \
                                      int grid_limit, int ntiles, cudaStream_t st) {                        \
    return launch_batch_t<S>(vset, bt, w, p, srows, amp, bstep, mask, stages, grid_limit, ntiles, st);    \
  }                                                                                                      \
  cudaError_t launch_moments_##SUF(int vset, const void *fin, const HostGeom &g, double eps0, double vmax2, \
                                   double *e, double *ux, double *uy, double *part, unsigned *err,       \
                                   dim3 b, cudaStream_t st) {                                            \
    return launch_moments_t<S>(vset, fin, g, eps0, vmax2, e, ux, uy, part, err, b, st);                  \
  }                                                                                                      \
  cudaError_t launch_init_##SUF(int vset, void *fout, const HostGeom &g, double eps0, const double *e,  \
                                const double *ux, const double *uy, cudaStream_t st) {                   \
    return launch_init_t<S>(vset, fout, g, eps0, e, ux, uy, st);                                         \
  }                                                                                                      \
  cudaError_t launch_ghosts_##SUF(int vset, void *f, const HostGeom &g, cudaStream_t st) {              \
    return launch_ghosts_t<S>(vset, f, g, st);                                                           \
  }                                                                                                      \
  cudaError_t launch_open_ghosts_##SUF(int vset, void *f, const HostGeom &g, double ux_in, cudaStream_t st) { \
    return launch_open_ghosts_t<S>(vset, f, g, ux_in, st);                                               \
  }                                                                                                      \
  cudaError_t launch_stir_prime_##SUF(const HostStir &s, void *cn, void *cn1, void *G, int nx,          \
                                      long long n, cudaStream_t st) {                                    \
    return launch_stir_prime_t<S>(s, cn, cn1, G, nx, n, st);                                             \
  }                                                                                                      \
  }
