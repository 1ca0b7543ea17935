// Host-side launch interface between the C ABI (rlbm_capi.cu) and the kernels of
// each storage type (rlbm_kernels_*.cu).  Plain structs, no templates.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rlbm {

// Boundary flags of a lattice (Geometry::walls): bit 0 = bounce-back walls in y (the ghost
// rows stay zero), bit 1 = open channel in x (inflow column left of x = 0, written once;
// zero-gradient outflow right of x = nx - 1), bit 2 = a strip of a larger lattice (the
// ghost rows are written by the halo exchange, never by the kernels; which ghost-row cells
// are solid is in the neighbour mask).
constexpr int WALLS_Y = 1, OPEN_X = 2, STRIP_Y = 4;

struct HostGeom {
  int nx, ny, pitch;
  long long plane;         // elements per ghost-padded plane: pitch * (ny + 2)
  int walls;
  const uint16_t *nbmask;  // device; NULL when the lattice has no solid cells or walls
  double beta[17][4];
};

struct HostPhys {
  double omega0, fpref, body_x, body_y, vmax2;
  int has_force;
  int stochastic;          // 16-bit storage: stochastic rounding
  unsigned round_key;      // key of the rounding bits
  long long step;          // index n of the step being launched
  int y_off;               // lattice row of the context's row 0 (a strip of a larger lattice; else 0)
};

struct HostStir {
  int nrows, nmodes;
  const void *G_cur, *EY;
  int eyp;
  void *G_next;
  const void *coef_next;
  void *coef_new;
  const int *mode_kx, *row_start;
  unsigned long long seed;
  long long step_new;
  double amp;
  const double *mode_scale;  // device [nmodes]; NULL = all 1
};

// One lattice of a batch, as the batched step kernel sees it (device memory, written by
// the host before the launches; 128-byte aligned so its tensor maps are 64-byte aligned).
struct alignas(128) MemberDesc {
  CUtensorMap tin[2];      // loads of population buffer 0 / 1
  CUtensorMap tG[2];       // stirring rows of step parity 0 / 1
  CUtensorMap tEY;
  void *f[2];              // population buffers
  const uint16_t *nbmask;  // NULL = no solid cells and no walls
  int nx, ny, pitch, walls;
  long long plane;
  int cur0;                // buffer holding f*_n at batch step 0
  int nrows, nmodes, eyp;
  long long step0;         // the member's step index at batch step 0
  const void *G[2], *EY, *coef[2];
  const int *mode_kx, *row_start;
  unsigned long long seed;
  unsigned round_key;
  unsigned *err;
  int ntx;                 // tiles per row
  float rcp_ntx;           // 1 / ntx (tile index -> row and column with one correction)
};

// Prefix tables of a batch (device): tiles, stirring-table entries and draws per member.
struct BatchTables {
  const MemberDesc *mem;
  const int *tile0;        // [n + 1]
  const long long *entry0; // [n + 1]
  const int *draw0;        // [n + 1]
  int *tile_ctr;           // tiles handed out so far in this launch (0 before each launch)
  int n;
};

#define RLBM_DECLARE_LAUNCHERS(SUF)                                                                      \
  cudaError_t launch_step_##SUF(int vset, const void *tin, const void *tg, const void *tey, void *fout,     \
                                const HostGeom &g, const HostPhys &p, const HostStir &s, unsigned *err, \
                                int grid_limit, int stages, int stir_rows, int *ctr, unsigned seq,      \
                                bool chained, void *macro_out, cudaStream_t st);                         \
  cudaError_t launch_ghosts_##SUF(int vset, void *f, const HostGeom &g, cudaStream_t st);               \
  cudaError_t launch_batch_step_##SUF(int vset, const BatchTables &bt, const HostGeom &w, const HostPhys &p, \
                                      int srows, double amp, const long long *bstep, bool mask, int stages, \
                                      int grid_limit, int ntiles, cudaStream_t st);                       \
  cudaError_t launch_moments_##SUF(int vset, const void *fin, const HostGeom &g, double eps0, double vmax2, \
                                   double *e, double *ux, double *uy, double *part, unsigned *err,       \
                                   dim3 b, cudaStream_t st);                                             \
  cudaError_t launch_init_##SUF(int vset, void *fout, const HostGeom &g, double eps0, const double *e,  \
                                const double *ux, const double *uy, cudaStream_t st);                   \
  cudaError_t launch_open_ghosts_##SUF(int vset, void *f, const HostGeom &g, double ux_in, cudaStream_t st); \
  cudaError_t launch_stir_prime_##SUF(const HostStir &s, void *cn, void *cn1, void *G, int nx,          \
                                      long long n, cudaStream_t st);

RLBM_DECLARE_LAUNCHERS(f64)
RLBM_DECLARE_LAUNCHERS(f32)
RLBM_DECLARE_LAUNCHERS(f16)
RLBM_DECLARE_LAUNCHERS(bf16)

// One adjoint step (rlbm_adjoint.cu): buffers and tables of the launch.
struct AdjointArgs {
  const void *B;           // post-collision buffer B_{n-1} (storage type)
  const void *kin;         // kappa_{n+1} (compute type), NULL for the last state
  const void *tB, *tK;     // host CUtensorMap load maps of B and kin (the layout of the state)
  bool chained;            // the launch directly follows the reverse step of step n + 1 on the
                           // stream, and B was written before that step (programmatic launch)
  const void *macro;       // the step's eps/eps0 - 1, v_x, v_y, F_x, F_y and streamed h_0 .. h_{Q-1}
                           // per cell from the forward recomputation (5 + Q planes of nx * ny), or
                           // NULL (then B is pulled and matched: the objective of the last state)
  void *kout;              // kappa_n
  double cj;               // objective weight of the state S_n
  double *acc;             // [blocks][4] FP64 accumulators
  void *zpart;             // [block rows][nrows][nx] R4 of the compute type (this step's slot)
  const void *G, *EY;      // stirring tables of step n
  int nrows, eyp;
  unsigned *err;
};
// The mode gradients of nj consecutive steps from their adjoint launches' row projections.
struct ModeGradArgs {
  const void *zpart;       // [nj][block rows][nrows][nx] R4 of the compute type
  void *zsum;              // [nj][nrows][nx] R4 of the compute type
  const void *tw;          // [nx] double2 exp(+2 pi i t / nx)
  const void *twf;         // [nx] float2, the same rounded to FP32
  int nj, nby, nrows, nx, nmodes;
  const int *mode_kx, *row_start;
  unsigned long long seed;
  long long n0;            // step index of j = 0
  double amp;
  double *gstep;           // [nj][nmodes] per-step d J / d sigma_m (this segment's rows)
};
cudaError_t launch_adjoint_f64(int vset, const AdjointArgs &a, const HostGeom &g, const HostPhys &p, cudaStream_t st);
cudaError_t launch_adjoint_f32(int vset, const AdjointArgs &a, const HostGeom &g, const HostPhys &p, cudaStream_t st);
cudaError_t launch_mode_grads_f64(const ModeGradArgs &a, cudaStream_t st);
cudaError_t launch_mode_grads_f32(const ModeGradArgs &a, cudaStream_t st);
cudaError_t launch_mode_sum(const double *gstep, long long nsteps, int nmodes, double *gsig, cudaStream_t st);
cudaError_t launch_adj_twiddles(double2 *tw, float2 *twf, int n, cudaStream_t st);

// Halo rows of a strip (rlbm_aux.cu): nplanes rows of row_bytes each, the plane p's row at
// byte offset off[p] of the population buffer, to (pack) or from (unpack) buf[p * row_bytes].
struct HaloRows {
  int nplanes;
  long long off[8];
};
cudaError_t launch_halo_copy(char *pop, const HaloRows &rows, long long row_bytes, char *buf, bool pack,
                             cudaStream_t st);

// Reductions and spectrum (rlbm_aux.cu)
cudaError_t launch_counter_inc(long long *counter, int *tile_ctr, cudaStream_t st);
cudaError_t launch_reduce_partials(const double *partials, long long nblocks, double *totals, cudaStream_t st);
cudaError_t launch_column_means(const double *ux, const double *uy, int nx, int ny, double *jx, double *jy,
                                cudaStream_t st);
cudaError_t launch_band_energy(const double *ux, const double *uy, int nx, int ny, const double2 *twx,
                               const double2 *twy, double2 *z0, double2 *z1, long long k2lo, long long k2hi,
                               double *partials, double *out4, cudaStream_t st);
cudaError_t launch_spectrum(const double *ux, const double *uy, int nx, int ny, const double2 *twx,
                            const double2 *twy, double2 *z0, double2 *z1, double *bins, int nbins,
                            cudaStream_t st);

}  // namespace rlbm
