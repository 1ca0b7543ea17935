// C ABI of the relativistic lattice Boltzmann library: configuration checks, the
// workspace layout in the caller's device memory, host-built tables (streaming
// weights, stirring modes and phase tables, FFT twiddles, solid-neighbour masks) and
// the dispatch of the kernels of each storage type.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rlbm.h"
#include "rlbm_device.cuh"
#include "rlbm_launch.h"

using namespace rlbm;

namespace {

thread_local std::string g_thread_error;

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int num_classes(int vset) { return vset == 3 ? VSet<3>::Q : VSet<2>::Q; }
size_t store_bytes(int prec) { return prec == RLBM_F64 ? 8 : prec == RLBM_F32 ? 4 : 2; }
size_t real_bytes(int prec) { return prec == RLBM_F64 ? 8 : 4; }

struct Modes {
  std::vector<int> kx, ky, row_start, row_ky;
};

// Half-plane integer wave vectors of the shell kmin^2 <= |k|^2 <= kmax^2, sorted by
// (k_y, k_x), grouped into rows of equal k_y.
Modes shell_modes(int kmin, int kmax) {
  Modes m;
  for (int ky = 0; ky <= kmax; ++ky)
    for (int kx = -kmax; kx <= kmax; ++kx) {
      const int k2 = kx * kx + ky * ky;
      if ((ky > 0 || kx > 0) && kmin * kmin <= k2 && k2 <= kmax * kmax) {
        if (m.row_ky.empty() || m.row_ky.back() != ky) {
          m.row_ky.push_back(ky);
          m.row_start.push_back((int)m.kx.size());
        }
        m.kx.push_back(kx);
        m.ky.push_back(ky);
      }
    }
  m.row_start.push_back((int)m.kx.size());
  return m;
}

bool stirring_on(const rlbm_config &c) { return c.force_amp != 0.0; }

// A strip of a larger lattice (rlbm_config::strip_ny_total > 0); its lattice's row count.
bool is_strip(const rlbm_config &c) { return c.strip_ny_total > 0; }
int total_rows(const rlbm_config &c) { return is_strip(c) ? c.strip_ny_total : c.ny; }
// Faces of a strip whose ghost rows come from a neighbour (bit 0: below row 0, bit 1: above
// row ny - 1); a face at the first or last row of a lattice with walls is a wall.
int halo_faces(const rlbm_config &c) {
  if (!is_strip(c)) return 0;
  int f = 3;
  if (c.walls_y && c.strip_y0 == 0) f &= ~1;
  if (c.walls_y && c.strip_y0 + c.ny == c.strip_ny_total) f &= ~2;
  return f;
}
bool needs_mask(const rlbm_config &c) { return c.solid || c.walls_y || (is_strip(c) && c.strip_solid_halo); }

struct Layout {
  size_t pop[2], nbmask, err, ctr, EY, G[2], coef[2], mode_kx, row_start, mode_scale;
  size_t eps, ux, uy, partials, totals, twx, twy, z0, z1, bins, cols, total;
  long long plane;
  int pitch, xoff, Q, nrows, nmodes, max_bins, eyp;
  long long max_blocks;
};

Layout make_layout(const rlbm_config &c) {
  Layout L{};
  L.Q = num_classes(c.vset);
  const size_t sb = store_bytes(c.precision), rb = real_bytes(c.precision);
  // ghost-padded planes: 128-byte left margin (interior starts on a line), one ghost
  // column each side, rows padded to whole 128-byte lines; one ghost row each side
  L.xoff = (int)(128 / sb);
  L.pitch = (int)((L.xoff + c.nx + 1 + L.xoff - 1) / L.xoff * L.xoff);
  L.plane = (long long)L.pitch * (c.ny + 2);
  const size_t ncell = (size_t)c.nx * c.ny;
  Modes m;
  if (stirring_on(c)) m = shell_modes(c.kmin, c.kmax);
  L.nmodes = (int)m.kx.size();
  L.nrows = (int)m.row_ky.size();
  L.max_blocks = (long long)((c.nx + 31) / 32) * c.ny;
  L.max_bins = (int)std::ceil(std::sqrt((c.nx / 2 + 1.0) * (c.nx / 2 + 1.0) + (c.ny / 2 + 1.0) * (c.ny / 2 + 1.0))) + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(std::max<size_t>(bytes, 1)); return o; };
  L.pop[0] = take(sb * L.Q * L.plane);
  L.pop[1] = take(sb * L.Q * L.plane);
  L.nbmask = take(needs_mask(c) ? 2 * ncell : 0);
  L.err = take(16);
  L.ctr = take(16);  // tile counters of the step kernel (two, used by alternate launches)
  L.eyp = (c.ny + 7) / 8 * 8;  // EY rows padded to 8 entries (16-byte TMA strides)
  L.EY = take(2 * rb * (size_t)L.nrows * L.eyp);
  L.G[0] = take(4 * rb * (size_t)L.nrows * c.nx);
  L.G[1] = take(4 * rb * (size_t)L.nrows * c.nx);
  L.coef[0] = take(4 * rb * L.nmodes);
  L.coef[1] = take(4 * rb * L.nmodes);
  L.mode_kx = take(4 * L.nmodes);
  L.row_start = take(4 * (L.nrows + 1));
  L.mode_scale = take(8 * L.nmodes);
  L.eps = take(8 * ncell);
  L.ux = take(8 * ncell);
  L.uy = take(8 * ncell);
  L.partials = take(32 * (size_t)std::max<long long>(L.max_blocks, c.nx));  // moments blocks, or one per k_x column
  L.totals = take(32);
  L.twx = take(16 * (size_t)c.nx);
  L.twy = take(16 * (size_t)c.ny);
  L.z0 = take(16 * ncell);
  L.z1 = take(16 * ncell);
  L.bins = take(8 * (size_t)L.max_bins);
  L.cols = take(16 * (size_t)c.nx);  // column means j_x, j_y
  L.total = off;
  return L;
}

std::string validate(const rlbm_config *c) {
  if (!c) return "cfg is NULL";
  if (c->nx < 8 || c->ny < 8 || c->nx > 32768 || c->ny > 32768) return "nx and ny must lie in [8, 32768]";
  if (c->walls_y != 0 && c->walls_y != 1) return "walls_y must be 0 or 1";
  if (c->vset != 2 && c->vset != 3) return "vset must be 2 or 3";
  if (c->precision < RLBM_F64 || c->precision > RLBM_BF16) return "precision must be one of RLBM_F64..RLBM_BF16";
  if (c->rounding != 0 && c->rounding != 1) return "rounding must be 0 (stochastic) or 1 (to nearest)";
  if (!(c->a > 0.0) || !(c->dt > 0.0) || !std::isfinite(c->a) || !std::isfinite(c->dt))
    return "a and dt must be positive and finite";
  if (c->dt / c->a > 1.0) return "dt / a must not exceed 1 (the streaming displacement stays within one cell)";
  if (!(c->eta_over_s > 0.0) || !std::isfinite(c->eta_over_s)) return "eta_over_s must be positive and finite";
  if (!(c->eps0 > 0.0) || !std::isfinite(c->eps0)) return "eps0 must be positive and finite";
  if (!std::isfinite(c->body_force[0]) || !std::isfinite(c->body_force[1])) return "body_force must be finite";
  if (!std::isfinite(c->force_amp)) return "force_amp must be finite";
  if (c->strip_ny_total < 0) return "strip_ny_total must be >= 0 (0: the context is the whole lattice)";
  if (is_strip(*c)) {
    if (c->strip_ny_total > (1 << 30)) return "strip_ny_total must not exceed 2^30";
    if (c->strip_y0 < 0 || (long long)c->strip_y0 + c->ny > c->strip_ny_total)
      return "a strip needs 0 <= strip_y0 and strip_y0 + ny <= strip_ny_total";
    if (c->open_x) return "a strip cannot be an open channel";
  }
  if (stirring_on(*c)) {
    if (c->kmin < 0 || c->kmax < c->kmin) return "the stirring shell needs 0 <= kmin <= kmax";
    if (2 * c->kmax >= std::min(c->nx, total_rows(*c))) return "kmax must be below min(nx, ny) / 2 (ny of the whole lattice)";
    if (shell_modes(c->kmin, c->kmax).kx.empty()) return "the stirring shell holds no wave vector";
  }
  if (c->vset == 2 && (stirring_on(*c) || c->body_force[0] != 0.0 || c->body_force[1] != 0.0))
    return "the projected force is defined for the three-dimensional momentum set (vset 3) only";
  if (!(c->fp64_landau_vmax >= 0.0 && c->fp64_landau_vmax < 1.0)) return "fp64_landau_vmax must lie in [0, 1)";
  if (c->open_x != 0 && c->open_x != 1) return "open_x must be 0 or 1";
  if (c->open_x && !(std::fabs(c->inflow_ux) < 1.0)) return "inflow_ux must be finite with |inflow_ux| < 1";
  return "";
}

double temperature_of(double eps, int vset) {
  return vset == 3 ? std::pow(M_PI * M_PI * eps / 3.0, 0.25) : std::cbrt(M_PI * eps);
}

template <int VS> void fill_beta(double C, double beta[17][4]) {
  for (int q = 0; q < VSet<VS>::Q; ++q) {
    const double ax = C * std::fabs(VSet<VS>::vx(q)), ay = C * std::fabs(VSet<VS>::vy(q));
    beta[q][0] = (1.0 - ax) * (1.0 - ay);
    beta[q][1] = ax * (1.0 - ay);
    beta[q][2] = (1.0 - ax) * ay;
    beta[q][3] = ax * ay;
  }
}

struct Scoped {  // switch to the context's device for one call, restore afterwards
  int prev = -1, want;
  explicit Scoped(int dev) : want(dev) {
    cudaGetDevice(&prev);
    if (prev != want) cudaSetDevice(want);
  }
  ~Scoped() {
    if (prev >= 0 && prev != want) cudaSetDevice(prev);
  }
};

}  // namespace

struct rlbm_ctx {
  rlbm_config cfg;
  Layout L;
  int device = 0;
  cudaStream_t stream = nullptr;
  char *ws = nullptr;
  int cur = 0;           // population buffer holding f*_n
  int64_t step = 0;
  long long nfluid = 0;  // cells that are not solid
  bool unit_scale = true;  // every stirring multiplier sigma_m is 1
  rlbm_status latched = RLBM_OK;
  std::string msg;
  HostGeom geom;
  HostPhys phys;
  dim3 block{32, 8, 1};       // moments kernel
  int grid_limit = 0;          // step kernel: 0 = one wave of resident CTAs
  int stages = 2;              // shared-memory pipeline depth of the step kernel (1 or 2)
  int stir_rows = 1;           // stirring rows: 1 = staged with each tile, 2 = read from global memory
  unsigned launch_seq = 0;     // step-kernel launches so far (selects the tile counter)
  int halo_faces = 0;          // a strip: faces whose ghost rows come from neighbours (bit 0 below, 1 above)
  int halo_pending = 0;        // faces not unpacked since the last step, set_state or init
  CUtensorMap tmap_in[2], tmap_G[2], tmap_EY;
  std::vector<uint8_t> host_stage;

  template <typename T> T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }

  rlbm_status fail(rlbm_status s, const std::string &m) {
    msg = m;
    return s;
  }
  rlbm_status cuda_fail(cudaError_t e, const char *what) {
    msg = std::string(what) + ": " + cudaGetErrorString(e);
    return RLBM_E_CUDA;
  }
};

namespace {

// Step n from the buffer behind `ti` into `fout`; its stirring rows come from s.G_cur and,
// when staged by TMA, through `tgmap` (NULL: the context's table of step parity n & 1).
// `chained`: the launch directly follows the step kernel of step n - 1 on the stream
// (programmatic dependent launch).  `macro_out` (compute type, 5 planes of nx * ny, may be
// NULL): each fluid cell's eps/eps0 - 1, v_x, v_y, F_x, F_y of the step, for the reverse sweep.
cudaError_t dispatch_step_raw(rlbm_ctx *c, const CUtensorMap *ti, void *fout, int64_t n, const HostStir &s,
                              const CUtensorMap *tgmap = nullptr, bool chained = false, void *macro_out = nullptr) {
  unsigned *err = c->at<unsigned>(c->L.err);
  const void *tg = tgmap ? tgmap : &c->tmap_G[n & 1], *te = &c->tmap_EY;
  int *ctr = c->at<int>(c->L.ctr);
  const unsigned seq = c->launch_seq++;
  switch (c->cfg.precision) {
    case RLBM_F64: return launch_step_f64(c->cfg.vset, ti, tg, te, fout, c->geom, c->phys, s, err, c->grid_limit, c->stages, c->stir_rows, ctr, seq, chained, macro_out, c->stream);
    case RLBM_F32: return launch_step_f32(c->cfg.vset, ti, tg, te, fout, c->geom, c->phys, s, err, c->grid_limit, c->stages, c->stir_rows, ctr, seq, chained, macro_out, c->stream);
    case RLBM_F16: return launch_step_f16(c->cfg.vset, ti, tg, te, fout, c->geom, c->phys, s, err, c->grid_limit, c->stages, c->stir_rows, ctr, seq, chained, macro_out, c->stream);
    default: return launch_step_bf16(c->cfg.vset, ti, tg, te, fout, c->geom, c->phys, s, err, c->grid_limit, c->stages, c->stir_rows, ctr, seq, chained, macro_out, c->stream);
  }
}

cudaError_t dispatch_step(rlbm_ctx *c, int src, const HostStir &s, bool chained = false) {
  return dispatch_step_raw(c, &c->tmap_in[src], c->ws + c->L.pop[src ^ 1], c->step, s, nullptr, chained);
}

cudaError_t dispatch_ghosts(rlbm_ctx *c, int b) {
  void *f = c->ws + c->L.pop[b];
  switch (c->cfg.precision) {
    case RLBM_F64: return launch_ghosts_f64(c->cfg.vset, f, c->geom, c->stream);
    case RLBM_F32: return launch_ghosts_f32(c->cfg.vset, f, c->geom, c->stream);
    case RLBM_F16: return launch_ghosts_f16(c->cfg.vset, f, c->geom, c->stream);
    default: return launch_ghosts_bf16(c->cfg.vset, f, c->geom, c->stream);
  }
}

// Inflow and outflow columns of an open channel (no-op for x periodic).
cudaError_t dispatch_open_ghosts(rlbm_ctx *c, int b) {
  if (!c->cfg.open_x) return cudaSuccess;
  void *f = c->ws + c->L.pop[b];
  const double u = c->cfg.inflow_ux;
  switch (c->cfg.precision) {
    case RLBM_F64: return launch_open_ghosts_f64(c->cfg.vset, f, c->geom, u, c->stream);
    case RLBM_F32: return launch_open_ghosts_f32(c->cfg.vset, f, c->geom, u, c->stream);
    case RLBM_F16: return launch_open_ghosts_f16(c->cfg.vset, f, c->geom, u, c->stream);
    default: return launch_open_ghosts_bf16(c->cfg.vset, f, c->geom, u, c->stream);
  }
}

// Tensor maps of one population buffer: the whole ghost-padded planes, {pitch, ny + 2,
// Q}, read in boxes of {32 + 2 V, 10, Q} (a 32 x 8 tile with its halo, V = 16 bytes of
// elements).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder() {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && fn) encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return encode;
}

// Load map of a population buffer at `base` (the layout of the context's own buffers).
std::string encode_state_map(const rlbm_ctx *c, void *base, CUtensorMap *out) {
  EncodeTiledFn encode = tensor_map_encoder();
  if (!encode) return "cuTensorMapEncodeTiled is not available";
  const int prec = c->cfg.precision;
  const size_t eb = store_bytes(prec);
  const CUtensorMapDataType dt = prec == RLBM_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : prec == RLBM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : prec == RLBM_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const cuuint32_t V = (cuuint32_t)(16 / eb);
  const cuuint64_t strides[2] = {(cuuint64_t)c->L.pitch * eb, (cuuint64_t)c->L.plane * eb};
  const cuuint32_t estr[3] = {1, 1, 1};
  const cuuint64_t din[3] = {(cuuint64_t)c->L.pitch, (cuuint64_t)c->cfg.ny + 2, (cuuint64_t)c->L.Q};
  const cuuint32_t bin[3] = {32 + 2 * V, 10, (cuuint32_t)c->L.Q};
  CUresult r = encode(out, dt, 3, base, din, strides, bin, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled (load map) failed with " + std::to_string((int)r);
  return "";
}

// Load map of a stirring-row table {nrows}{nx} R4 at `base` (staged shells, nrows <= 16).
std::string encode_table_map(const rlbm_ctx *c, void *base, CUtensorMap *out) {
  EncodeTiledFn encode = tensor_map_encoder();
  if (!encode) return "cuTensorMapEncodeTiled is not available";
  const int prec = c->cfg.precision;
  const CUtensorMapDataType rt = prec == RLBM_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const size_t rb = real_bytes(prec);
  const cuuint32_t e2[2] = {1, 1};
  const cuuint64_t dg[2] = {(cuuint64_t)4 * c->cfg.nx, (cuuint64_t)c->L.nrows};
  const cuuint64_t sg[1] = {(cuuint64_t)4 * c->cfg.nx * rb};
  const cuuint32_t bg[2] = {4 * 32, (cuuint32_t)c->L.nrows};
  CUresult r = encode(out, rt, 2, base, dg, sg, bg, e2, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled (stirring table map) failed with " + std::to_string((int)r);
  return "";
}

std::string make_tensor_maps(rlbm_ctx *c) {
  EncodeTiledFn encode = tensor_map_encoder();
  if (!encode) return "cuTensorMapEncodeTiled is not available";
  const int prec = c->cfg.precision;
  for (int b = 0; b < 2; ++b) {
    const std::string m = encode_state_map(c, c->ws + c->L.pop[b], &c->tmap_in[b]);
    if (!m.empty()) return m;
  }
  // stirring tables of a tile: G rows {4 nx} (one R4 per column) in boxes {4 * 32, nrows},
  // EY rows {2 eyp} in boxes {2 * 8, nrows}; staged only for shells of <= 16 k_y rows
  std::memset(c->tmap_G, 0, sizeof(c->tmap_G));
  std::memset(&c->tmap_EY, 0, sizeof(c->tmap_EY));
  if (c->L.nrows > 0 && c->L.nrows <= 16) {
    const CUtensorMapDataType rt = prec == RLBM_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const size_t rb = real_bytes(prec);
    const cuuint32_t e2[2] = {1, 1};
    for (int b = 0; b < 2; ++b) {
      const std::string m = encode_table_map(c, c->ws + c->L.G[b], &c->tmap_G[b]);
      if (!m.empty()) return m;
    }
    const cuuint64_t de[2] = {(cuuint64_t)2 * c->L.eyp, (cuuint64_t)c->L.nrows};
    const cuuint64_t se[1] = {(cuuint64_t)2 * c->L.eyp * rb};
    const cuuint32_t be[2] = {2 * 8, (cuuint32_t)c->L.nrows};
    CUresult r = encode(&c->tmap_EY, rt, 2, c->ws + c->L.EY, de, se, be, e2, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled (phase table map) failed with " + std::to_string((int)r);
  }
  return "";
}

cudaError_t dispatch_moments(rlbm_ctx *c) {
  const void *fin = c->ws + c->L.pop[c->cur];
  double *e = c->at<double>(c->L.eps), *ux = c->at<double>(c->L.ux), *uy = c->at<double>(c->L.uy);
  double *part = c->at<double>(c->L.partials);
  unsigned *err = c->at<unsigned>(c->L.err);
  const double e0 = c->cfg.eps0;
  cudaError_t r;
  switch (c->cfg.precision) {
    case RLBM_F64: r = launch_moments_f64(c->cfg.vset, fin, c->geom, e0, c->phys.vmax2, e, ux, uy, part, err, c->block, c->stream); break;
    case RLBM_F32: r = launch_moments_f32(c->cfg.vset, fin, c->geom, e0, c->phys.vmax2, e, ux, uy, part, err, c->block, c->stream); break;
    case RLBM_F16: r = launch_moments_f16(c->cfg.vset, fin, c->geom, e0, c->phys.vmax2, e, ux, uy, part, err, c->block, c->stream); break;
    default: r = launch_moments_bf16(c->cfg.vset, fin, c->geom, e0, c->phys.vmax2, e, ux, uy, part, err, c->block, c->stream); break;
  }
  if (r != cudaSuccess) return r;
  const long long nblocks = (long long)((c->cfg.nx + c->block.x - 1) / c->block.x) * ((c->cfg.ny + c->block.y - 1) / c->block.y);
  return launch_reduce_partials(part, nblocks, c->at<double>(c->L.totals), c->stream);
}

cudaError_t dispatch_init(rlbm_ctx *c, void *fout, const double *e, const double *ux, const double *uy) {
  switch (c->cfg.precision) {
    case RLBM_F64: return launch_init_f64(c->cfg.vset, fout, c->geom, c->cfg.eps0, e, ux, uy, c->stream);
    case RLBM_F32: return launch_init_f32(c->cfg.vset, fout, c->geom, c->cfg.eps0, e, ux, uy, c->stream);
    case RLBM_F16: return launch_init_f16(c->cfg.vset, fout, c->geom, c->cfg.eps0, e, ux, uy, c->stream);
    default: return launch_init_bf16(c->cfg.vset, fout, c->geom, c->cfg.eps0, e, ux, uy, c->stream);
  }
}

HostStir stir_for_step(rlbm_ctx *c, int64_t n) {
  HostStir s{};
  const Layout &L = c->L;
  s.nrows = L.nrows;
  s.nmodes = L.nmodes;
  if (L.nmodes == 0) return s;
  s.G_cur = c->ws + L.G[n & 1];
  s.G_next = c->ws + L.G[(n + 1) & 1];
  s.coef_next = c->ws + L.coef[(n + 1) & 1];
  s.coef_new = c->ws + L.coef[n & 1];
  s.EY = c->ws + L.EY;
  s.eyp = L.eyp;
  s.mode_kx = c->at<int>(L.mode_kx);
  s.row_start = c->at<int>(L.row_start);
  s.seed = c->cfg.seed;
  s.step_new = n + 2;
  s.amp = c->cfg.force_amp;
  s.mode_scale = c->unit_scale ? nullptr : c->at<double>(L.mode_scale);
  return s;
}

// Coefficients of steps n and n+1 and the table of step n.
cudaError_t stir_prime(rlbm_ctx *c, int64_t n) {
  if (c->L.nmodes == 0) return cudaSuccess;
  HostStir s = stir_for_step(c, n);
  void *cn = c->ws + c->L.coef[n & 1], *cn1 = c->ws + c->L.coef[(n + 1) & 1], *G = c->ws + c->L.G[n & 1];
  switch (c->cfg.precision) {
    case RLBM_F64: return launch_stir_prime_f64(s, cn, cn1, G, c->cfg.nx, n, c->stream);
    case RLBM_F32: return launch_stir_prime_f32(s, cn, cn1, G, c->cfg.nx, n, c->stream);
    case RLBM_F16: return launch_stir_prime_f16(s, cn, cn1, G, c->cfg.nx, n, c->stream);
    default: return launch_stir_prime_bf16(s, cn, cn1, G, c->cfg.nx, n, c->stream);
  }
}

// Reads the device error word after a synchronisation and latches it.
rlbm_status check_device(rlbm_ctx *c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "cudaStreamSynchronize");
  unsigned w = 0;
  e = cudaMemcpy(&w, c->at<unsigned>(c->L.err), sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return c->cuda_fail(e, "cudaMemcpy(error word)");
  if (w & ERR_UNSTABLE) {
    c->latched = RLBM_E_UNSTABLE;
    return c->fail(RLBM_E_UNSTABLE, "a cell became non-finite, eps <= 0 or |v| >= 1 (numerically unstable run)");
  }
  if (w & ERR_UNPHYSICAL) {
    c->latched = RLBM_E_UNPHYSICAL;
    return c->fail(RLBM_E_UNPHYSICAL, "Landau matching found no timelike eigenvector in some cell");
  }
  if (w & ERR_TIMEOUT) {
    c->latched = RLBM_E_TIMEOUT;
    return c->fail(RLBM_E_TIMEOUT, "a bounded device-side wait expired (a copy did not complete in time); "
                                   "the results of the queued work are incomplete");
  }
  return RLBM_OK;
}

rlbm_status usable(rlbm_ctx *c) {
  if (c->latched != RLBM_OK) {
    c->msg = "the context is in an error state (" + std::to_string((int)c->latched) + "); only rlbm_free is allowed";
    return RLBM_E_STATE;
  }
  return RLBM_OK;
}

// h of a stored value and back (FP16 storage holds HScale<__half>::up times h)
template <typename S> double to_double(S v) { return (double)v; }
template <> double to_double<__half>(__half v) { return (double)__half2float(v) * HScale<__half>::down; }
template <> double to_double<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <typename S> S from_double(double v) { return (S)v; }
template <> __half from_double<__half>(double v) { return __float2half_rn((float)(v * HScale<__half>::up)); }
template <> __nv_bfloat16 from_double<__nv_bfloat16>(double v) { return __float2bfloat16_rn((float)v); }

template <typename S> void unpack_state(const rlbm_ctx *c, const uint8_t *src, double *dst) {
  const S *p = reinterpret_cast<const S *>(src);
  const int nx = c->cfg.nx, ny = c->cfg.ny;
  for (int q = 0; q < c->L.Q; ++q)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        dst[((size_t)q * ny + y) * nx + x] = to_double<S>(p[q * c->L.plane + (size_t)(y + 1) * c->L.pitch + x + c->L.xoff]);
}

template <typename S> void pack_state(const rlbm_ctx *c, const double *src, uint8_t *dst) {
  S *p = reinterpret_cast<S *>(dst);
  const int nx = c->cfg.nx, ny = c->cfg.ny;
  for (int q = 0; q < c->L.Q; ++q)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        p[q * c->L.plane + (size_t)(y + 1) * c->L.pitch + x + c->L.xoff] = from_double<S>(src[((size_t)q * ny + y) * nx + x]);
}

}  // namespace

namespace rlbm {
// Lets the allocation-free entry point (rlbm_noalloc.cu) report through rlbm_last_error(NULL).
void set_thread_error(const std::string &msg) { g_thread_error = msg; }
// The bounded-wait self-test kernel (rlbm_aux.cu).
cudaError_t launch_wait_selftest(unsigned *err, long long max_cycles, cudaStream_t st);
}  // namespace rlbm

extern "C" {

rlbm_status rlbm_query_workspace(const rlbm_config *cfg, size_t *bytes) {
  const std::string v = validate(cfg);
  if (!v.empty()) { g_thread_error = v; return RLBM_E_INVAL; }
  if (!bytes) { g_thread_error = "bytes is NULL"; return RLBM_E_INVAL; }
  *bytes = make_layout(*cfg).total;
  return RLBM_OK;
}

rlbm_status rlbm_init(const rlbm_config *cfg, void *dev_workspace, size_t bytes, void *cuda_stream, rlbm_ctx **out) {
  if (!out) { g_thread_error = "out is NULL"; return RLBM_E_INVAL; }
  *out = nullptr;
  const std::string v = validate(cfg);
  if (!v.empty()) { g_thread_error = v; return RLBM_E_INVAL; }
  const Layout L = make_layout(*cfg);
  if (!dev_workspace) { g_thread_error = "dev_workspace is NULL"; return RLBM_E_INVAL; }
  if (reinterpret_cast<uintptr_t>(dev_workspace) % kAlign) { g_thread_error = "dev_workspace must be 256-byte aligned"; return RLBM_E_INVAL; }
  if (bytes < L.total) {
    g_thread_error = "workspace too small: " + std::to_string(bytes) + " < " + std::to_string(L.total) + " bytes";
    return RLBM_E_NOMEM;
  }
  const size_t ncell = (size_t)cfg->nx * cfg->ny;
  // host-side checks of the initial fields
  for (size_t i = 0; cfg->init_eps && i < ncell; ++i)
    if (!(cfg->init_eps[i] > 0.0) || !std::isfinite(cfg->init_eps[i])) { g_thread_error = "init_eps must be positive and finite"; return RLBM_E_INVAL; }
  for (size_t i = 0; i < ncell; ++i) {
    const double a = cfg->init_ux ? cfg->init_ux[i] : 0.0, b = cfg->init_uy ? cfg->init_uy[i] : 0.0;
    if (!std::isfinite(a) || !std::isfinite(b)) { g_thread_error = "init_ux / init_uy must be finite"; return RLBM_E_INVAL; }
  }

  rlbm_ctx *c = new (std::nothrow) rlbm_ctx();
  if (!c) { g_thread_error = "host allocation failed"; return RLBM_E_NOMEM; }
  c->cfg = *cfg;
  c->cfg.solid = nullptr; c->cfg.init_eps = c->cfg.init_ux = c->cfg.init_uy = nullptr;
  c->cfg.strip_solid_halo = nullptr;
  c->halo_faces = c->halo_pending = halo_faces(*cfg);
  c->L = L;
  c->ws = static_cast<char *>(dev_workspace);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&c->device);
  if (c->cfg.fp64_landau_vmax == 0.0) c->cfg.fp64_landau_vmax = 0.5;

  auto bail = [&](rlbm_status s) { g_thread_error = c->msg; delete c; return s; };
  auto put = [&](size_t off, const void *src, size_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    return cudaMemcpyAsync(c->ws + off, src, n, cudaMemcpyHostToDevice, c->stream);
  };

  // streaming weights
  const double C = cfg->dt / cfg->a;
  std::memset(c->geom.beta, 0, sizeof(c->geom.beta));
  if (cfg->vset == 3) fill_beta<3>(C, c->geom.beta); else fill_beta<2>(C, c->geom.beta);
  c->geom.nx = cfg->nx; c->geom.ny = cfg->ny; c->geom.pitch = L.pitch; c->geom.plane = L.plane;
  c->geom.walls = is_strip(*cfg) ? STRIP_Y : (cfg->walls_y ? WALLS_Y : 0) | (cfg->open_x ? OPEN_X : 0);
  c->geom.nbmask = nullptr;
  {
    const std::string tm = make_tensor_maps(c);
    if (!tm.empty()) { c->msg = tm; return bail(RLBM_E_CUDA); }
  }

  // relaxation and force constants
  const double T0 = temperature_of(cfg->eps0, cfg->vset);
  const double taunum = cfg->vset == 3 ? VSet<3>::TAU_NUM : VSet<2>::TAU_NUM;
  c->phys.omega0 = cfg->dt * T0 / (taunum * cfg->eta_over_s);
  c->phys.fpref = -6.0 * cfg->dt / T0;
  c->phys.body_x = cfg->body_force[0];
  c->phys.body_y = cfg->body_force[1];
  c->phys.vmax2 = c->cfg.fp64_landau_vmax * c->cfg.fp64_landau_vmax;
  c->phys.has_force = (stirring_on(*cfg) || cfg->body_force[0] != 0.0 || cfg->body_force[1] != 0.0) ? 1 : 0;
  c->phys.stochastic = cfg->rounding == 0 ? 1 : 0;
  c->phys.round_key = (unsigned)(cfg->seed ^ (cfg->seed >> 32)) ^ 0x5bd1e995u;
  c->phys.y_off = is_strip(*cfg) ? cfg->strip_y0 : 0;

  // Host staging buffers; copies from pageable memory have consumed their source when
  // cudaMemcpyAsync returns, and init synchronises the stream before it returns.
  std::vector<std::vector<uint8_t>> keep;
  cudaError_t e = cudaSuccess;

  c->nfluid = (long long)ncell;
  for (size_t i = 0; cfg->solid && i < ncell; ++i)
    if (cfg->solid[i] != 0) --c->nfluid;

  // solid-neighbour masks: bit 4 = the cell, bit (dy+1)*3+(dx+1) = neighbour (x+dx, y+dy);
  // rows y = -1 and y = ny are solid when walls_y is set.  For a strip, a ghost row is solid
  // at a wall face, and elsewhere as strip_solid_halo says.
  if (needs_mask(*cfg)) {
    keep.emplace_back(2 * ncell);
    uint16_t *nb = reinterpret_cast<uint16_t *>(keep.back().data());
    const int nx = cfg->nx, ny = cfg->ny;
    const int faces = halo_faces(*cfg);
    auto solid_at = [&](int x, int y) -> bool {
      if (is_strip(*cfg) && (y < 0 || y >= ny)) {
        const int face = y < 0 ? 0 : 1;
        if (!(faces & (1 << face))) return true;  // a wall
        x = (x + nx) % nx;
        return cfg->strip_solid_halo && cfg->strip_solid_halo[(size_t)face * nx + x] != 0;
      }
      if (y < 0 || y >= ny) {
        if (cfg->walls_y) return true;
        y = (y + ny) % ny;
      }
      if (cfg->open_x && (x < 0 || x >= nx)) return false;  // inflow / outflow columns
      x = (x + nx) % nx;
      return cfg->solid && cfg->solid[(size_t)y * nx + x] != 0;
    };
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        uint16_t m = 0;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx)
            if (solid_at(x + dx, y + dy)) m |= (uint16_t)(1u << ((dy + 1) * 3 + (dx + 1)));
        nb[(size_t)y * nx + x] = m;
      }
    if ((e = put(L.nbmask, nb, 2 * ncell)) != cudaSuccess) { c->cuda_fail(e, "upload of the solid mask"); return bail(RLBM_E_CUDA); }
    c->geom.nbmask = c->at<uint16_t>(L.nbmask);
  }

  // stirring tables (library's own; FP64-built, stored in the compute type)
  if (L.nmodes) {
    const Modes m = shell_modes(cfg->kmin, cfg->kmax);
    // phase rows in the layout of ey_index: per row 2 eyp reals, blocks of 8 lattice rows,
    // entry k of a block = (Re y, Re y+1, Im y, Im y+1) for y = 8 b + 2 k
    // (the phase of lattice row y0 + y for a strip starting at row y0 of ny_t rows)
    std::vector<double> ey((size_t)L.nrows * 2 * L.eyp, 0.0);
    const long long y0 = is_strip(*cfg) ? cfg->strip_y0 : 0, nyt = total_rows(*cfg);
    for (int r = 0; r < L.nrows; ++r)
      for (int y = 0; y < cfg->ny; ++y) {
        const long long j = ((long long)m.row_ky[r] * (y0 + y)) % nyt;
        const size_t i = (size_t)r * 2 * L.eyp + ey_index(y);
        ey[i] = std::cos(2.0 * M_PI * (double)j / (double)nyt);
        ey[i + 2] = std::sin(2.0 * M_PI * (double)j / (double)nyt);
      }
    keep.emplace_back();
    if (cfg->precision == RLBM_F64) {
      keep.back().resize(ey.size() * sizeof(double));
      std::memcpy(keep.back().data(), ey.data(), ey.size() * sizeof(double));
    } else {
      keep.back().resize(ey.size() * sizeof(float));
      float *pf = reinterpret_cast<float *>(keep.back().data());
      for (size_t i = 0; i < ey.size(); ++i) pf[i] = (float)ey[i];
    }
    const std::vector<double> ones(L.nmodes, 1.0);
    keep.emplace_back(reinterpret_cast<const uint8_t *>(ones.data()), reinterpret_cast<const uint8_t *>(ones.data()) + 8 * ones.size());
    if ((e = put(L.mode_scale, keep.back().data(), keep.back().size())) != cudaSuccess ||
        (e = put(L.EY, keep[keep.size() - 2].data(), keep[keep.size() - 2].size())) != cudaSuccess ||
        (e = put(L.mode_kx, m.kx.data(), 4 * m.kx.size())) != cudaSuccess ||
        (e = put(L.row_start, m.row_start.data(), 4 * m.row_start.size())) != cudaSuccess) {
      c->cuda_fail(e, "upload of the stirring tables");
      return bail(RLBM_E_CUDA);
    }
  }

  // FFT twiddles exp(-2 pi i t / n)
  {
    std::vector<double> twx(2 * (size_t)cfg->nx), twy(2 * (size_t)cfg->ny);
    for (int t = 0; t < cfg->nx; ++t) { twx[2 * t] = std::cos(2.0 * M_PI * t / cfg->nx); twx[2 * t + 1] = -std::sin(2.0 * M_PI * t / cfg->nx); }
    for (int t = 0; t < cfg->ny; ++t) { twy[2 * t] = std::cos(2.0 * M_PI * t / cfg->ny); twy[2 * t + 1] = -std::sin(2.0 * M_PI * t / cfg->ny); }
    keep.emplace_back(reinterpret_cast<uint8_t *>(twx.data()), reinterpret_cast<uint8_t *>(twx.data()) + 16 * (size_t)cfg->nx);
    keep.emplace_back(reinterpret_cast<uint8_t *>(twy.data()), reinterpret_cast<uint8_t *>(twy.data()) + 16 * (size_t)cfg->ny);
    if ((e = put(L.twx, keep[keep.size() - 2].data(), 16 * (size_t)cfg->nx)) != cudaSuccess ||
        (e = put(L.twy, keep.back().data(), 16 * (size_t)cfg->ny)) != cudaSuccess) {
      c->cuda_fail(e, "upload of the FFT twiddles");
      return bail(RLBM_E_CUDA);
    }
  }

  // initial fields -> f*_0 = f_eq in both population buffers
  const double *de = nullptr, *dux = nullptr, *duy = nullptr;
  if (cfg->init_eps) { if ((e = put(L.eps, cfg->init_eps, 8 * ncell)) != cudaSuccess) { c->cuda_fail(e, "upload of init_eps"); return bail(RLBM_E_CUDA); } de = c->at<double>(L.eps); }
  if (cfg->init_ux) { if ((e = put(L.ux, cfg->init_ux, 8 * ncell)) != cudaSuccess) { c->cuda_fail(e, "upload of init_ux"); return bail(RLBM_E_CUDA); } dux = c->at<double>(L.ux); }
  if (cfg->init_uy) { if ((e = put(L.uy, cfg->init_uy, 8 * ncell)) != cudaSuccess) { c->cuda_fail(e, "upload of init_uy"); return bail(RLBM_E_CUDA); } duy = c->at<double>(L.uy); }
  for (int b = 0; b < 2; ++b) {
    if ((e = cudaMemsetAsync(c->ws + L.pop[b], 0, store_bytes(cfg->precision) * L.Q * L.plane, c->stream)) != cudaSuccess) {
      c->cuda_fail(e, "cudaMemsetAsync");
      return bail(RLBM_E_CUDA);
    }
    if ((e = dispatch_init(c, c->ws + L.pop[b], de, dux, duy)) != cudaSuccess) { c->cuda_fail(e, "init kernel"); return bail(RLBM_E_CUDA); }
    if ((e = dispatch_open_ghosts(c, b)) != cudaSuccess) { c->cuda_fail(e, "open-channel ghost kernel"); return bail(RLBM_E_CUDA); }
  }
  if ((e = cudaMemsetAsync(c->ws + L.err, 0, 16, c->stream)) != cudaSuccess) { c->cuda_fail(e, "cudaMemsetAsync"); return bail(RLBM_E_CUDA); }
  if ((e = cudaMemsetAsync(c->ws + L.ctr, 0, 16, c->stream)) != cudaSuccess) { c->cuda_fail(e, "cudaMemsetAsync"); return bail(RLBM_E_CUDA); }
  if ((e = stir_prime(c, 0)) != cudaSuccess) { c->cuda_fail(e, "stirring set-up kernels"); return bail(RLBM_E_CUDA); }
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) { c->cuda_fail(e, "cudaStreamSynchronize"); return bail(RLBM_E_CUDA); }
  c->cur = 0;
  c->step = 0;
  *out = c;
  return RLBM_OK;
}

rlbm_status rlbm_step(rlbm_ctx *c, int64_t nsteps) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (nsteps < 0) return c->fail(RLBM_E_INVAL, "nsteps must be >= 0");
  if (c->halo_faces && nsteps > 0) {
    if (nsteps > 1) return c->fail(RLBM_E_INVAL, "a strip steps one step at a time, between halo exchanges");
    if (c->halo_pending) return c->fail(RLBM_E_STATE, "the strip's ghost rows are not unpacked since its last step");
    c->halo_pending = c->halo_faces;
  }
  Scoped dev(c->device);
  for (int64_t i = 0; i < nsteps; ++i) {
    const HostStir s = stir_for_step(c, c->step);
    c->phys.step = c->step;
    cudaError_t e = dispatch_step(c, c->cur, s, i > 0);
    if (e != cudaSuccess) return c->cuda_fail(e, "step kernel launch");
    c->cur ^= 1;
    ++c->step;
  }
  return RLBM_OK;
}

rlbm_status rlbm_moments(rlbm_ctx *c, double *eps, double *ux, double *uy, double *totals) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (c->halo_pending) return c->fail(RLBM_E_STATE, "the strip's ghost rows are not unpacked since its last step");
  Scoped dev(c->device);
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny * sizeof(double);
  cudaError_t e = dispatch_moments(c);
  if (e != cudaSuccess) return c->cuda_fail(e, "moments kernel launch");
  if (eps && (e = cudaMemcpyAsync(eps, c->ws + c->L.eps, n, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of eps");
  if (ux && (e = cudaMemcpyAsync(ux, c->ws + c->L.ux, n, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of ux");
  if (uy && (e = cudaMemcpyAsync(uy, c->ws + c->L.uy, n, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of uy");
  if (totals && (e = cudaMemcpyAsync(totals, c->ws + c->L.totals, 32, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of totals");
  return check_device(c);
}

rlbm_status rlbm_spectrum(rlbm_ctx *c, int32_t nbins, double *E) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (is_strip(c->cfg)) return c->fail(RLBM_E_INVAL, "a strip has no spectrum of its own: it needs the whole lattice");
  if (nbins < 1 || !E) return c->fail(RLBM_E_INVAL, "nbins must be >= 1 and E non-NULL");
  Scoped dev(c->device);
  cudaError_t e = dispatch_moments(c);
  if (e != cudaSuccess) return c->cuda_fail(e, "moments kernel launch");
  const int nb = std::min(nbins, c->L.max_bins);
  e = launch_spectrum(c->at<double>(c->L.ux), c->at<double>(c->L.uy), c->cfg.nx, c->cfg.ny,
                      c->at<double2>(c->L.twx), c->at<double2>(c->L.twy), c->at<double2>(c->L.z0),
                      c->at<double2>(c->L.z1), c->at<double>(c->L.bins), nb, c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "spectrum kernels");
  if ((e = cudaMemcpyAsync(E, c->ws + c->L.bins, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return c->cuda_fail(e, "copy of the spectrum");
  rlbm_status s = check_device(c);
  for (int i = nb; i < nbins; ++i) E[i] = 0.0;  // beyond the largest |k| of the lattice
  return s;
}

rlbm_status rlbm_get_state(rlbm_ctx *c, double *host, int64_t *step) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (!host) return c->fail(RLBM_E_INVAL, "host is NULL");
  Scoped dev(c->device);
  const size_t bytes = store_bytes(c->cfg.precision) * c->L.Q * c->L.plane;
  c->host_stage.resize(bytes);
  cudaError_t e = cudaMemcpyAsync(c->host_stage.data(), c->ws + c->L.pop[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "copy of the state");
  rlbm_status s = check_device(c);
  if (s != RLBM_OK) return s;
  switch (c->cfg.precision) {
    case RLBM_F64: unpack_state<double>(c, c->host_stage.data(), host); break;
    case RLBM_F32: unpack_state<float>(c, c->host_stage.data(), host); break;
    case RLBM_F16: unpack_state<__half>(c, c->host_stage.data(), host); break;
    default: unpack_state<__nv_bfloat16>(c, c->host_stage.data(), host); break;
  }
  if (step) *step = c->step;
  return RLBM_OK;
}

rlbm_status rlbm_set_state(rlbm_ctx *c, const double *host, int64_t step) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (!host || step < 0) return c->fail(RLBM_E_INVAL, "host must be non-NULL and step >= 0");
  Scoped dev(c->device);
  const size_t bytes = store_bytes(c->cfg.precision) * c->L.Q * c->L.plane;
  c->host_stage.assign(bytes, 0);
  switch (c->cfg.precision) {
    case RLBM_F64: pack_state<double>(c, host, c->host_stage.data()); break;
    case RLBM_F32: pack_state<float>(c, host, c->host_stage.data()); break;
    case RLBM_F16: pack_state<__half>(c, host, c->host_stage.data()); break;
    default: pack_state<__nv_bfloat16>(c, host, c->host_stage.data()); break;
  }
  cudaError_t e = cudaMemcpyAsync(c->ws + c->L.pop[c->cur], c->host_stage.data(), bytes, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "copy of the state");
  c->step = step;
  c->halo_pending = c->halo_faces;
  if ((e = dispatch_ghosts(c, c->cur)) != cudaSuccess) return c->cuda_fail(e, "ghost fill kernel");
  if ((e = dispatch_open_ghosts(c, c->cur)) != cudaSuccess) return c->cuda_fail(e, "open-channel ghost kernel");
  if ((e = stir_prime(c, step)) != cudaSuccess) return c->cuda_fail(e, "stirring set-up kernels");
  return check_device(c);
}

rlbm_status rlbm_band_energy(rlbm_ctx *c, int64_t k2lo, int64_t k2hi, double *E) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (is_strip(c->cfg)) return c->fail(RLBM_E_INVAL, "a strip has no band energy of its own: it needs the whole lattice");
  if (!E || k2lo < 0) return c->fail(RLBM_E_INVAL, "E must be non-NULL and k2lo >= 0");
  Scoped dev(c->device);
  cudaError_t e = dispatch_moments(c);
  if (e != cudaSuccess) return c->cuda_fail(e, "moments kernel launch");
  double *out = c->at<double>(c->L.totals);
  e = launch_band_energy(c->at<double>(c->L.ux), c->at<double>(c->L.uy), c->cfg.nx, c->cfg.ny,
                         c->at<double2>(c->L.twx), c->at<double2>(c->L.twy), c->at<double2>(c->L.z0),
                         c->at<double2>(c->L.z1), k2lo, k2hi, c->at<double>(c->L.partials), out, c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "band energy kernels");
  double host[4];
  if ((e = cudaMemcpyAsync(host, out, 32, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of the band energy");
  if (rlbm_status s = check_device(c)) return s;
  *E = host[0];
  return RLBM_OK;
}

rlbm_status rlbm_column_means(rlbm_ctx *c, double *jx, double *jy) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (is_strip(c->cfg)) return c->fail(RLBM_E_INVAL, "a strip has no column means of its own: it needs the whole lattice");
  Scoped dev(c->device);
  cudaError_t e = dispatch_moments(c);
  if (e != cudaSuccess) return c->cuda_fail(e, "moments kernel launch");
  double *d = c->at<double>(c->L.cols);
  const int nx = c->cfg.nx;
  if ((e = launch_column_means(c->at<double>(c->L.ux), c->at<double>(c->L.uy), nx, c->cfg.ny, d, d + nx, c->stream)) != cudaSuccess)
    return c->cuda_fail(e, "column means kernel");
  if (jx && (e = cudaMemcpyAsync(jx, d, 8 * (size_t)nx, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of j_x");
  if (jy && (e = cudaMemcpyAsync(jy, d + nx, 8 * (size_t)nx, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of j_y");
  return check_device(c);
}

}  // extern "C"

namespace {

// The planes that cross a face and the byte offsets of their boundary or ghost rows in the
// current population buffer.  Moving down (v_y < 0) crosses face 0 from above: the strip
// below needs row 0's such planes in its ghost row above (unpack face 1), and this strip's
// ghost row below (unpack face 0) receives the planes moving up.
HaloRows halo_rows(const rlbm_ctx *c, int face, bool pack) {
  HaloRows h{};
  const int Q = c->L.Q;
  const int want = (face == 0) == pack ? -1 : 1;  // sign of v_y of the planes carried
  const long long row = pack ? (face == 0 ? 1 : c->cfg.ny) : (face == 0 ? 0 : c->cfg.ny + 1);
  const long long sb = (long long)store_bytes(c->cfg.precision);
  for (int q = 0; q < Q; ++q) {
    const double vy = c->cfg.vset == 3 ? VSet<3>::vy(q) : VSet<2>::vy(q);
    if ((vy > 1e-12 ? 1 : vy < -1e-12 ? -1 : 0) != want) continue;
    h.off[h.nplanes++] = sb * ((long long)q * c->L.plane + row * c->L.pitch);
  }
  return h;
}

rlbm_status halo_copy(rlbm_ctx *c, int32_t face, void *dev, bool pack) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (!is_strip(c->cfg)) return c->fail(RLBM_E_INVAL, "the context is a whole lattice, not a strip");
  if (face != 0 && face != 1) return c->fail(RLBM_E_INVAL, "face must be 0 (below row 0) or 1 (above row ny - 1)");
  if (!(c->halo_faces & (1 << face))) return c->fail(RLBM_E_INVAL, "that face of the strip is a wall");
  if (!dev || reinterpret_cast<uintptr_t>(dev) % 16) return c->fail(RLBM_E_INVAL, "the halo buffer must be a 16-byte aligned device pointer");
  Scoped d(c->device);
  const HaloRows h = halo_rows(c, face, pack);
  const long long row_bytes = (long long)store_bytes(c->cfg.precision) * c->L.pitch;
  cudaError_t e = launch_halo_copy(c->ws + c->L.pop[c->cur], h, row_bytes, static_cast<char *>(dev), pack, c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, pack ? "halo pack kernel" : "halo unpack kernel");
  if (!pack) c->halo_pending &= ~(1 << face);
  return RLBM_OK;
}

}  // namespace

extern "C" {

rlbm_status rlbm_halo_bytes(const rlbm_ctx *c, size_t *bytes) {
  if (!c || !bytes) { g_thread_error = "ctx and bytes must be non-NULL"; return RLBM_E_INVAL; }
  *bytes = is_strip(c->cfg) ? (size_t)halo_rows(c, 0, true).nplanes * store_bytes(c->cfg.precision) * c->L.pitch : 0;
  return RLBM_OK;
}

rlbm_status rlbm_halo_pack(rlbm_ctx *c, int32_t face, void *dev_out) { return halo_copy(c, face, dev_out, true); }

rlbm_status rlbm_halo_unpack(rlbm_ctx *c, int32_t face, const void *dev_in) {
  return halo_copy(c, face, const_cast<void *>(dev_in), false);
}

int32_t rlbm_num_planes(const rlbm_ctx *c) { return c ? c->L.Q : -1; }

int32_t rlbm_velocity_classes(int32_t vset, double *out) {
  if (vset != 2 && vset != 3) return -1;
  const int Q = num_classes(vset);
  for (int q = 0; out && q < Q; ++q) {
    out[4 * q + 0] = vset == 3 ? VSet<3>::vx(q) : VSet<2>::vx(q);
    out[4 * q + 1] = vset == 3 ? VSet<3>::vy(q) : VSet<2>::vy(q);
    out[4 * q + 2] = vset == 3 ? VSet<3>::vz2(q) : VSet<2>::vz2(q);
    out[4 * q + 3] = vset == 3 ? VSet<3>::w(q) : VSet<2>::w(q);
  }
  return Q;
}

rlbm_status rlbm_set_launch(rlbm_ctx *c, int32_t ctas, int32_t stages, int32_t stir_rows) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (ctas < 0 || stages < 0 || stages > 2 || stir_rows < 0 || stir_rows > 2)
    return c->fail(RLBM_E_INVAL, "ctas must be >= 0, stages 0, 1 or 2 and stir_rows 0, 1 or 2");
  c->grid_limit = ctas;
  if (stages) c->stages = stages;
  if (stir_rows) c->stir_rows = stir_rows;
  return RLBM_OK;
}

rlbm_status rlbm_autotune(rlbm_ctx *c, int32_t reps, double *ms_out) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (reps < 1) return c->fail(RLBM_E_INVAL, "reps must be >= 1");
  Scoped dev(c->device);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  // candidate launch shapes: pipeline depth x persistent CTA count (0 = all resident) x
  // where the stirring rows come from (staged with each tile, or global memory)
  const int stage_opts[2] = {2, 1};
  const int grid_opts[4] = {0, 2 * sms, 3 * sms, 4 * sms};
  const int rows_opts[2] = {1, 2};
  const int nrows_opts = (c->L.nrows > 0 && c->L.nrows <= 16) ? 2 : 1;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return c->fail(RLBM_E_CUDA, "cudaEventCreate failed");
  const int save_grid = c->grid_limit, save_stages = c->stages, save_rows = c->stir_rows;
  float best = 1e30f;
  int best_grid = save_grid, best_stages = save_stages, best_rows = save_rows;
  const HostStir st = stir_for_step(c, c->step);
  cudaError_t e = cudaSuccess;
  for (int ri = 0; ri < nrows_opts && e == cudaSuccess; ++ri)
    for (int si = 0; si < 2 && e == cudaSuccess; ++si)
      for (int gi = 0; gi < 4 && e == cudaSuccess; ++gi) {
        c->stir_rows = rows_opts[ri];
        c->stages = stage_opts[si];
        c->grid_limit = grid_opts[gi];
        // the step kernel reads the current buffer and writes the other one; repeating it
        // leaves the state (and the step counter) as it was.  The repetitions are chained as
        // rlbm_step chains consecutive steps (programmatic dependent launch), so the shape is
        // chosen for the way the steps run.
        if ((e = dispatch_step(c, c->cur, st)) != cudaSuccess) break;  // warm-up
        cudaEventRecord(e0, c->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = dispatch_step(c, c->cur, st, r > 0);
        cudaEventRecord(e1, c->stream);
        if (e != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_grid = c->grid_limit; best_stages = c->stages; best_rows = c->stir_rows; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->grid_limit = best_grid;
  c->stages = best_stages;
  c->stir_rows = best_rows;
  if (e != cudaSuccess) {
    c->grid_limit = save_grid; c->stages = save_stages; c->stir_rows = save_rows;
    return c->cuda_fail(e, "autotune launch");
  }
  if (ms_out) *ms_out = best / reps;
  return check_device(c);
}

rlbm_status rlbm_wait_selftest(rlbm_ctx *c, int64_t max_cycles) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (max_cycles < 1 || max_cycles > (int64_t(1) << 31))
    return c->fail(RLBM_E_INVAL, "max_cycles must lie in [1, 2^31]");
  Scoped dev(c->device);
  const cudaError_t e = launch_wait_selftest(c->at<unsigned>(c->L.err), max_cycles, c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "self-test kernel launch");
  return RLBM_OK;
}

rlbm_status rlbm_sync(rlbm_ctx *c) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  Scoped dev(c->device);
  return check_device(c);
}

int64_t rlbm_current_step(const rlbm_ctx *c) { return c ? c->step : -1; }

const char *rlbm_last_error(const rlbm_ctx *c) { return c ? c->msg.c_str() : g_thread_error.c_str(); }

void rlbm_free(rlbm_ctx *c) {
  if (!c) return;
  {
    Scoped dev(c->device);
    cudaStreamSynchronize(c->stream);
  }
  delete c;
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
}  // extern "C"

struct rlbm_batch {
  std::vector<rlbm_ctx *> members;
  char *ws = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  MemberDesc *d_mem = nullptr;
  int *d_tile0 = nullptr, *d_draw0 = nullptr;
  long long *d_entry0 = nullptr, *d_bstep = nullptr;
  int *d_tctr = nullptr;  // the batched kernel's tile counter
  std::vector<MemberDesc> h_mem;
  int ntiles = 0, srows = 0, stages = 2, grid_limit = 0;
  bool mask = false;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  std::string msg;
  rlbm_status fail(rlbm_status s, const std::string &m) { msg = m; return s; }
  rlbm_status cuda_fail(cudaError_t e, const char *what) { msg = std::string(what) + ": " + cudaGetErrorString(e); return RLBM_E_CUDA; }
};

namespace {

struct BatchLayout { size_t mem, tile0, entry0, draw0, bstep, tctr, total; };

BatchLayout batch_layout(int n) {
  BatchLayout L{};
  size_t off = 0;
  auto take = [&](size_t b) { size_t o = off; off += align_up(std::max<size_t>(b, 1)); return o; };
  L.mem = take(sizeof(MemberDesc) * (size_t)n);
  L.tile0 = take(sizeof(int) * (size_t)(n + 1));
  L.entry0 = take(sizeof(long long) * (size_t)(n + 1));
  L.draw0 = take(sizeof(int) * (size_t)(n + 1));
  L.bstep = take(sizeof(long long));
  L.tctr = take(sizeof(int));
  L.total = off;
  return L;
}

bool same_physics(const rlbm_config &a, const rlbm_config &b) {
  return a.vset == b.vset && a.precision == b.precision && a.a == b.a && a.dt == b.dt &&
         a.eta_over_s == b.eta_over_s && a.eps0 == b.eps0 && a.body_force[0] == b.body_force[0] &&
         a.body_force[1] == b.body_force[1] && a.kmin == b.kmin && a.kmax == b.kmax && a.force_amp == b.force_amp &&
         a.rounding == b.rounding && a.fp64_landau_vmax == b.fp64_landau_vmax;
}

// The member table as the batched kernel reads it: every member's current buffer and
// step (members may have been stepped on their own), and the batch step counter at 0.
cudaError_t batch_prepare(rlbm_batch *b) {
  for (size_t i = 0; i < b->members.size(); ++i) {
    b->h_mem[i].cur0 = b->members[i]->cur;
    b->h_mem[i].step0 = b->members[i]->step;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_mem, b->h_mem.data(), sizeof(MemberDesc) * b->h_mem.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bstep, 0, sizeof(long long), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_tctr, 0, sizeof(int), b->stream);
  return e;
}

cudaError_t batch_launch_one(rlbm_batch *b) {
  rlbm_ctx *c0 = b->members[0];
  BatchTables bt{b->d_mem, b->d_tile0, b->d_entry0, b->d_draw0, b->d_tctr, (int)b->members.size()};
  cudaError_t e;
  const double amp = c0->cfg.force_amp;
  switch (c0->cfg.precision) {
    case RLBM_F64: e = launch_batch_step_f64(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream); break;
    case RLBM_F32: e = launch_batch_step_f32(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream); break;
    case RLBM_F16: e = launch_batch_step_f16(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream); break;
    default: e = launch_batch_step_bf16(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream); break;
  }
  if (e != cudaSuccess) return e;
  return launch_counter_inc(b->d_bstep, b->d_tctr, b->stream);
}

}  // namespace

extern "C" {

rlbm_status rlbm_batch_query_workspace(int32_t nmembers, size_t *bytes) {
  if (nmembers < 1 || !bytes) { g_thread_error = "nmembers must be >= 1 and bytes non-NULL"; return RLBM_E_INVAL; }
  *bytes = batch_layout(nmembers).total;
  return RLBM_OK;
}

rlbm_status rlbm_batch_init(rlbm_ctx *const *members, int32_t nmembers, void *dev_workspace, size_t bytes,
                            void *cuda_stream, rlbm_batch **out) {
  if (!out) { g_thread_error = "out is NULL"; return RLBM_E_INVAL; }
  *out = nullptr;
  if (!members || nmembers < 1) { g_thread_error = "members must hold nmembers >= 1 contexts"; return RLBM_E_INVAL; }
  const BatchLayout L = batch_layout(nmembers);
  if (!dev_workspace || reinterpret_cast<uintptr_t>(dev_workspace) % kAlign) { g_thread_error = "dev_workspace must be a 256-byte aligned device pointer"; return RLBM_E_INVAL; }
  if (bytes < L.total) { g_thread_error = "batch workspace too small"; return RLBM_E_NOMEM; }
  for (int i = 0; i < nmembers; ++i) {
    if (!members[i]) { g_thread_error = "member " + std::to_string(i) + " is NULL"; return RLBM_E_INVAL; }
    if (members[i]->latched != RLBM_OK) { g_thread_error = "member " + std::to_string(i) + " is in an error state"; return RLBM_E_STATE; }
    if (!same_physics(members[0]->cfg, members[i]->cfg))
      { g_thread_error = "member " + std::to_string(i) + " differs from member 0 in velocity set, storage type, a, dt, eta/s, eps0, force or rounding"; return RLBM_E_INVAL; }
    if (members[i]->device != members[0]->device) { g_thread_error = "members live on different devices"; return RLBM_E_INVAL; }
    if (members[i]->cfg.open_x) { g_thread_error = "member " + std::to_string(i) + " is an open channel (batches take periodic-x lattices)"; return RLBM_E_INVAL; }
    if (is_strip(members[i]->cfg)) { g_thread_error = "member " + std::to_string(i) + " is a strip (batches take whole lattices)"; return RLBM_E_INVAL; }
  }
  rlbm_batch *b = new (std::nothrow) rlbm_batch();
  if (!b) { g_thread_error = "host allocation failed"; return RLBM_E_NOMEM; }
  b->members.assign(members, members + nmembers);
  b->ws = static_cast<char *>(dev_workspace);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->device = members[0]->device;
  b->d_mem = reinterpret_cast<MemberDesc *>(b->ws + L.mem);
  b->d_tile0 = reinterpret_cast<int *>(b->ws + L.tile0);
  b->d_entry0 = reinterpret_cast<long long *>(b->ws + L.entry0);
  b->d_draw0 = reinterpret_cast<int *>(b->ws + L.draw0);
  b->d_bstep = reinterpret_cast<long long *>(b->ws + L.bstep);
  b->d_tctr = reinterpret_cast<int *>(b->ws + L.tctr);
  b->stages = members[0]->stages;
  const int nrows = members[0]->L.nrows;
  b->srows = (nrows > 0 && nrows <= 16) ? nrows : 0;
  std::vector<int> tile0(nmembers + 1, 0), draw0(nmembers + 1, 0);
  std::vector<long long> entry0(nmembers + 1, 0);
  b->h_mem.resize(nmembers);
  for (int i = 0; i < nmembers; ++i) {
    rlbm_ctx *c = members[i];
    MemberDesc &d = b->h_mem[i];
    std::memset(&d, 0, sizeof(d));
    d.tin[0] = c->tmap_in[0]; d.tin[1] = c->tmap_in[1];
    d.tG[0] = c->tmap_G[0]; d.tG[1] = c->tmap_G[1]; d.tEY = c->tmap_EY;
    d.f[0] = c->ws + c->L.pop[0]; d.f[1] = c->ws + c->L.pop[1];
    d.nbmask = c->geom.nbmask;
    d.nx = c->cfg.nx; d.ny = c->cfg.ny; d.pitch = c->L.pitch; d.walls = c->cfg.walls_y; d.plane = c->L.plane;
    d.nrows = c->L.nrows; d.nmodes = c->L.nmodes; d.eyp = c->L.eyp;
    d.G[0] = c->ws + c->L.G[0]; d.G[1] = c->ws + c->L.G[1]; d.EY = c->ws + c->L.EY;
    d.coef[0] = c->ws + c->L.coef[0]; d.coef[1] = c->ws + c->L.coef[1];
    d.mode_kx = c->at<int>(c->L.mode_kx); d.row_start = c->at<int>(c->L.row_start);
    d.seed = c->cfg.seed; d.round_key = c->phys.round_key; d.err = c->at<unsigned>(c->L.err);
    d.ntx = (c->cfg.nx + 31) / 32;
    d.rcp_ntx = 1.0f / (float)d.ntx;
    const int nt = d.ntx * ((c->cfg.ny + 7) / 8);
    tile0[i + 1] = tile0[i] + nt;
    entry0[i + 1] = entry0[i] + (c->L.nmodes ? (long long)c->L.nrows * c->cfg.nx : 0);
    draw0[i + 1] = draw0[i] + c->L.nmodes;
    if (c->geom.nbmask) b->mask = true;
  }
  b->ntiles = tile0[nmembers];
  Scoped dev(b->device);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(b->d_tile0, tile0.data(), sizeof(int) * (nmembers + 1), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_entry0, entry0.data(), sizeof(long long) * (nmembers + 1), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(b->d_draw0, draw0.data(), sizeof(int) * (nmembers + 1), cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
      (e = batch_prepare(b)) != cudaSuccess || (e = cudaStreamSynchronize(b->stream)) != cudaSuccess) {
    g_thread_error = std::string("batch tables upload: ") + cudaGetErrorString(e);
    delete b;
    return RLBM_E_CUDA;
  }
  *out = b;
  return RLBM_OK;
}

rlbm_status rlbm_batch_set_launch(rlbm_batch *b, int32_t ctas, int32_t stages) {
  if (!b) { g_thread_error = "batch is NULL"; return RLBM_E_INVAL; }
  if (ctas < 0 || stages < 0 || stages > 2) return b->fail(RLBM_E_INVAL, "ctas must be >= 0 and stages 0, 1 or 2");
  b->grid_limit = ctas;
  if (stages) b->stages = stages;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; b->graph_steps = 0; }
  return RLBM_OK;
}

rlbm_status rlbm_batch_autotune(rlbm_batch *b, int32_t reps, double *ms_out) {
  if (!b) { g_thread_error = "batch is NULL"; return RLBM_E_INVAL; }
  if (reps < 1) return b->fail(RLBM_E_INVAL, "reps must be >= 1");
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i]->latched != RLBM_OK) return b->fail(RLBM_E_STATE, "member " + std::to_string(i) + " is in an error state");
  Scoped dev(b->device);
  // the trial launches read the member table of the members' current states
  if (cudaError_t e0_ = batch_prepare(b); e0_ != cudaSuccess) return b->cuda_fail(e0_, "batch descriptor upload");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  BatchTables bt{b->d_mem, b->d_tile0, b->d_entry0, b->d_draw0, b->d_tctr, (int)b->members.size()};
  rlbm_ctx *c0 = b->members[0];
  const double amp = c0->cfg.force_amp;
  // one batched step without advancing the step counter: every member's next buffer and
  // next-step tables are rewritten with the same values, so repeating it changes nothing
  // (the tile counter is cleared before each trial, as the counter kernel does between steps)
  auto trial = [&]() -> cudaError_t {
    if (cudaError_t me = cudaMemsetAsync(b->d_tctr, 0, sizeof(int), b->stream); me != cudaSuccess) return me;
    switch (c0->cfg.precision) {
      case RLBM_F64: return launch_batch_step_f64(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream);
      case RLBM_F32: return launch_batch_step_f32(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream);
      case RLBM_F16: return launch_batch_step_f16(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream);
      default: return launch_batch_step_bf16(c0->cfg.vset, bt, c0->geom, c0->phys, b->srows, amp, b->d_bstep, b->mask, b->stages, b->grid_limit, b->ntiles, b->stream);
    }
  };
  const int stage_opts[2] = {2, 1};
  const int grid_opts[5] = {0, sms, 2 * sms, 3 * sms, 4 * sms};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return b->fail(RLBM_E_CUDA, "cudaEventCreate failed");
  const int save_grid = b->grid_limit, save_stages = b->stages;
  float best = 1e30f;
  int best_grid = save_grid, best_stages = save_stages;
  cudaError_t e = cudaSuccess;
  for (int si = 0; si < 2 && e == cudaSuccess; ++si)
    for (int gi = 0; gi < 5 && e == cudaSuccess; ++gi) {
      b->stages = stage_opts[si];
      b->grid_limit = grid_opts[gi];
      if ((e = trial()) != cudaSuccess) break;  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r) e = trial();
      cudaEventRecord(e1, b->stream);
      if (e != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_grid = b->grid_limit; best_stages = b->stages; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->grid_limit = e == cudaSuccess ? best_grid : save_grid;
  b->stages = e == cudaSuccess ? best_stages : save_stages;
  if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; b->graph_steps = 0; }
  if (e != cudaSuccess) return b->cuda_fail(e, "batch autotune launch");
  if (ms_out) *ms_out = best / reps;
  // device errors (if any) surface through the members' next syncing call
  return RLBM_OK;
}

rlbm_status rlbm_batch_step(rlbm_batch *b, int64_t nsteps) {
  if (!b) { g_thread_error = "batch is NULL"; return RLBM_E_INVAL; }
  if (nsteps < 0) return b->fail(RLBM_E_INVAL, "nsteps must be >= 0");
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i]->latched != RLBM_OK) return b->fail(RLBM_E_STATE, "member " + std::to_string(i) + " is in an error state");
  if (nsteps == 0) return RLBM_OK;
  Scoped dev(b->device);
  cudaError_t e = batch_prepare(b);
  if (e != cudaSuccess) return b->cuda_fail(e, "batch descriptor upload");
  // Whole chunks of steps replay one captured CUDA graph (kernel + counter advance per
  // step); the remainder, and any run on the legacy default stream (which cannot be
  // captured), launch directly.
  const int chunk = 64;
  int64_t done = 0;
  if (b->stream != nullptr && nsteps >= chunk) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      for (int i = 0; e == cudaSuccess && i < chunk; ++i) e = batch_launch_one(b);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return b->cuda_fail(e, "batch graph capture");
      b->graph_steps = chunk;
    }
    for (; done + chunk <= nsteps; done += chunk)
      if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return b->cuda_fail(e, "batch graph launch");
  }
  for (; done < nsteps; ++done)
    if ((e = batch_launch_one(b)) != cudaSuccess) return b->cuda_fail(e, "batch step launch");
  for (rlbm_ctx *c : b->members) {
    c->step += nsteps;
    c->cur ^= (int)(nsteps & 1);
  }
  return RLBM_OK;
}

const char *rlbm_batch_last_error(const rlbm_batch *b) { return b ? b->msg.c_str() : g_thread_error.c_str(); }

void rlbm_batch_free(rlbm_batch *b) {
  if (!b) return;
  {
    Scoped dev(b->device);
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
  }
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Stirring multipliers and the adjoint (gradient of the kinetic-energy objective)
// ---------------------------------------------------------------------------
namespace {

struct GradLayout {
  int64_t N;
  int seg, K, nslots;
  size_t state_bytes, kap_bytes, table_bytes, zpart_bytes;
  size_t ckpt, slots, kap[2], acc, gst, zpart, zsum, tw, twf, gstep, gsig, out, macro, scratch, gscratch, total;
  size_t macro_bytes;
  long long nblocks;
  int nby;
};

GradLayout grad_layout(const rlbm_ctx *c, int64_t N, int32_t segment) {
  GradLayout G{};
  G.N = N;
  G.seg = segment > 0 ? segment : std::max(1, (int)std::ceil(std::sqrt((double)N)));
  if (G.seg > N) G.seg = (int)N;
  G.K = (int)((N + G.seg - 1) / G.seg);
  G.nslots = std::min(2, G.seg - 1);  // ping-pong states of a segment's recomputation
  const int prec = c->cfg.precision;
  const size_t rb = real_bytes(prec);
  G.state_bytes = align_up(store_bytes(prec) * c->L.Q * c->L.plane);
  G.kap_bytes = align_up(rb * c->L.Q * c->L.plane);
  G.nby = (c->cfg.ny + 7) / 8;
  G.nblocks = (long long)((c->cfg.nx + 31) / 32) * G.nby;
  G.table_bytes = align_up(4 * rb * (size_t)c->L.nrows * c->cfg.nx);
  G.zpart_bytes = 4 * rb * (size_t)G.nby * c->L.nrows * c->cfg.nx;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(std::max<size_t>(bytes, 1)); return o; };
  G.ckpt = take(G.state_bytes * G.K);
  G.slots = take(G.state_bytes * G.nslots);
  G.kap[0] = take(G.kap_bytes);
  G.kap[1] = take(G.kap_bytes);
  G.acc = take(32 * (size_t)G.nblocks);
  G.gst = take(G.table_bytes * G.seg);                       // stirring rows of a segment's steps
  G.zpart = take(G.zpart_bytes * G.seg);                     // force-adjoint row projections
  G.zsum = take(4 * rb * (size_t)c->L.nrows * c->cfg.nx * G.seg);
  G.tw = take(16 * (size_t)c->cfg.nx);
  G.twf = take(8 * (size_t)c->cfg.nx);
  G.gstep = take(8 * (size_t)c->L.nmodes * (size_t)N);
  G.gsig = take(8 * (size_t)c->L.nmodes);
  G.out = take(64);
  // each recomputed step's eps/eps0 - 1, v_x, v_y, F_x, F_y and streamed h_q per cell, for the
  // reverse sweep
  G.macro_bytes = align_up((5 + (size_t)c->L.Q) * rb * (size_t)c->cfg.nx * c->cfg.ny);
  G.macro = take(G.macro_bytes * G.seg);
  G.scratch = take(G.state_bytes);   // output of the last recomputed step of a segment (unused)
  G.gscratch = take(G.table_bytes);  // and the stirring rows it prepares for the next step
  G.total = off;
  return G;
}

std::string grad_check(const rlbm_ctx *c, int64_t nsteps, int32_t segment) {
  if (c->cfg.precision != RLBM_F64 && c->cfg.precision != RLBM_F32)
    return "the adjoint runs on FP64 and FP32 storage (the 16-bit forms round stochastically)";
  if (c->cfg.open_x) return "the adjoint is built for periodic-x lattices (no open-channel boundaries)";
  if (is_strip(c->cfg)) return "the adjoint runs on a whole lattice, not on a strip";
  if (nsteps < 1) return "nsteps must be >= 1";
  if (segment < 0) return "segment must be >= 0 (0 = ceil(sqrt(nsteps)))";
  return "";
}

// The adjoint always takes the force path on the paper's set, so that dJ/dF_body is the
// derivative at F = 0 too (the forward with F = 0 is the same either way).
cudaError_t dispatch_adjoint(rlbm_ctx *c, const AdjointArgs &a) {
  HostPhys ph = c->phys;
  ph.has_force = c->cfg.vset == 3 ? 1 : 0;
  if (c->cfg.precision == RLBM_F64) return launch_adjoint_f64(c->cfg.vset, a, c->geom, ph, c->stream);
  return launch_adjoint_f32(c->cfg.vset, a, c->geom, ph, c->stream);
}

}  // namespace

extern "C" {

int32_t rlbm_num_modes(const rlbm_ctx *c) { return c ? c->L.nmodes : -1; }

rlbm_status rlbm_set_mode_scale(rlbm_ctx *c, const double *sigma, int32_t nmodes) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  if (nmodes != c->L.nmodes) return c->fail(RLBM_E_INVAL, "nmodes must equal rlbm_num_modes(ctx) = " + std::to_string(c->L.nmodes));
  if (nmodes == 0) return RLBM_OK;
  if (!sigma) return c->fail(RLBM_E_INVAL, "sigma is NULL");
  bool unit = true;
  for (int m = 0; m < nmodes; ++m) {
    if (!std::isfinite(sigma[m])) return c->fail(RLBM_E_INVAL, "sigma must be finite");
    unit = unit && sigma[m] == 1.0;
  }
  Scoped dev(c->device);
  cudaError_t e = cudaMemcpyAsync(c->ws + c->L.mode_scale, sigma, 8 * (size_t)nmodes, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return c->cuda_fail(e, "copy of the mode multipliers");
  c->unit_scale = unit;
  // the coefficients and table of the current and next step are redrawn with them
  if ((e = stir_prime(c, c->step)) != cudaSuccess) return c->cuda_fail(e, "stirring set-up kernels");
  return check_device(c);
}

rlbm_status rlbm_gradient_query_workspace(const rlbm_ctx *c, int64_t nsteps, int32_t segment, size_t *bytes) {
  if (!c || !bytes) { g_thread_error = "ctx and bytes must be non-NULL"; return RLBM_E_INVAL; }
  const std::string m = grad_check(c, nsteps, segment);
  if (!m.empty()) { g_thread_error = m; return RLBM_E_INVAL; }
  *bytes = grad_layout(c, nsteps, segment).total;
  return RLBM_OK;
}

rlbm_status rlbm_gradient(rlbm_ctx *c, int64_t nsteps, int32_t segment, void *dev_workspace, size_t bytes, double *J,
                          double *grad_sigma, double *grad_eta_over_s, double *grad_body_force) {
  if (!c) { g_thread_error = "ctx is NULL"; return RLBM_E_INVAL; }
  if (rlbm_status s = usable(c)) return s;
  {
    const std::string m = grad_check(c, nsteps, segment);
    if (!m.empty()) return c->fail(RLBM_E_INVAL, m);
  }
  const GradLayout G = grad_layout(c, nsteps, segment);
  if (!dev_workspace || reinterpret_cast<uintptr_t>(dev_workspace) % kAlign)
    return c->fail(RLBM_E_INVAL, "dev_workspace must be a 256-byte aligned device pointer");
  if (bytes < G.total) return c->fail(RLBM_E_NOMEM, "gradient workspace too small: " + std::to_string(bytes) + " < " + std::to_string(G.total));
  if (c->nfluid < 1) return c->fail(RLBM_E_INVAL, "the lattice has no fluid cell");
  Scoped dev(c->device);
  char *w = static_cast<char *>(dev_workspace);
  auto ckpt = [&](int k) { return w + G.ckpt + G.state_bytes * (size_t)k; };
  auto slot = [&](int j) { return w + G.slots + G.state_bytes * (size_t)j; };
  std::vector<CUtensorMap> mck(G.K), msl(G.nslots);
  for (int k = 0; k < G.K; ++k) {
    const std::string m = encode_state_map(c, ckpt(k), &mck[k]);
    if (!m.empty()) return c->fail(RLBM_E_CUDA, m);
  }
  for (int j = 0; j < G.nslots; ++j) {
    const std::string m = encode_state_map(c, slot(j), &msl[j]);
    if (!m.empty()) return c->fail(RLBM_E_CUDA, m);
  }
  // load maps of the two adjoint buffers (compute type = storage type: FP32 or FP64)
  CUtensorMap mkap[2];
  for (int i = 0; i < 2; ++i) {
    const std::string m = encode_state_map(c, w + G.kap[i], &mkap[i]);
    if (!m.empty()) return c->fail(RLBM_E_CUDA, m);
  }
  auto gtab = [&](int j) { return w + G.gst + G.table_bytes * (size_t)j; };
  // the load maps of the per-step stirring rows are encoded as the steps are queued (not
  // all before the first launch), so that the host work overlaps the GPU's
  const bool staged_rows = c->L.nrows > 0 && c->L.nrows <= 16;
  std::string map_error;
  cudaError_t e;
  // Zeroed before use: the state and adjoint buffers (ghost rows of wall-bounded lattices
  // are never written) and the tile accumulators (added to), which lie together from ckpt up
  // to the stirring-row store, and the scratch state.  Everything else in the workspace is
  // written before it is read (the stored per-step values of a cell only where it is fluid,
  // and only those are read), so the tens of GB of one-segment runs are not cleared.
  if ((e = cudaMemsetAsync(w + G.ckpt, 0, G.gst - G.ckpt, c->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(w + G.scratch, 0, G.state_bytes, c->stream)) != cudaSuccess)
    return c->cuda_fail(e, "cudaMemsetAsync");

  // forward: B_{-1} (the context's buffer) to checkpoint 0; B_{k seg - 1} into checkpoint k.
  // With one segment the recomputation of that segment (below) is the forward itself: it
  // starts from checkpoint 0 and keeps every state, so no separate forward pass runs.
  const int64_t s0 = c->step;
  const bool one_pass = G.K == 1;
  if ((e = cudaMemcpyAsync(ckpt(0), c->ws + c->L.pop[c->cur], G.state_bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
    return c->cuda_fail(e, "copy of the start state");
  int where = -1;  // B_{n-1}: -1 - k = checkpoint k, 0 / 1 = context buffer
  for (int64_t n = 0; !one_pass && n < nsteps; ++n) {
    const CUtensorMap *ti = where < 0 ? &mck[-1 - where] : &c->tmap_in[where];
    void *fout;
    int next;
    if ((n + 1) % G.seg == 0 && n + 1 < nsteps) {
      next = -1 - (int)((n + 1) / G.seg);
      fout = ckpt((int)((n + 1) / G.seg));
    } else {
      next = where < 0 ? 0 : (where ^ 1);
      fout = c->ws + c->L.pop[next];
    }
    c->phys.step = s0 + n;
    if ((e = dispatch_step_raw(c, ti, fout, s0 + n, stir_for_step(c, s0 + n), nullptr, n > 0)) != cudaSuccess)
      return c->cuda_fail(e, "step kernel launch");
    where = next;
  }
  if (!one_pass) {
    c->cur = where;  // the last step writes a context buffer
    c->step = s0 + nsteps;
  }

  // reverse sweep
  if ((e = launch_adj_twiddles(reinterpret_cast<double2 *>(w + G.tw), reinterpret_cast<float2 *>(w + G.twf), c->cfg.nx,
                               c->stream)) != cudaSuccess)
    return c->cuda_fail(e, "twiddle kernel");
  AdjointArgs a{};
  a.acc = reinterpret_cast<double *>(w + G.acc);
  a.EY = c->ws + c->L.EY;
  a.nrows = c->L.nrows;
  a.eyp = c->L.eyp;
  a.err = c->at<unsigned>(c->L.err);
  ModeGradArgs mg{};
  mg.zpart = w + G.zpart;
  mg.zsum = w + G.zsum;
  mg.tw = w + G.tw;
  mg.twf = w + G.twf;
  mg.nby = G.nby;
  mg.nrows = c->L.nrows;
  mg.nx = c->cfg.nx;
  mg.nmodes = c->L.nmodes;
  mg.mode_kx = c->at<int>(c->L.mode_kx);
  mg.row_start = c->at<int>(c->L.row_start);
  mg.seed = c->cfg.seed;
  mg.amp = c->cfg.force_amp;
  double *gstep = reinterpret_cast<double *>(w + G.gstep), *gsig = reinterpret_cast<double *>(w + G.gsig);
  const double cj = 1.0 / ((double)nsteps * (double)c->nfluid);
  // stirring rows of steps lo .. hi-1 of segment k into the segment's table store, and each
  // step's stored values (Landau solution, force, streamed h) into its slot of G.macro; the
  // states B_lo .. B_{hi-2} alternate between the two ping-pong slots (B_{hi-1} goes to the
  // scratch state)
  auto recompute = [&](int k, int64_t lo, int64_t hi) -> cudaError_t {
    cudaError_t e2;
    if (c->L.nmodes) {
      HostStir sp = stir_for_step(c, s0 + lo);
      void *cn = c->ws + c->L.coef[(s0 + lo) & 1], *cn1 = c->ws + c->L.coef[(s0 + lo + 1) & 1];
      e2 = c->cfg.precision == RLBM_F64 ? launch_stir_prime_f64(sp, cn, cn1, gtab(0), c->cfg.nx, s0 + lo, c->stream)
                                        : launch_stir_prime_f32(sp, cn, cn1, gtab(0), c->cfg.nx, s0 + lo, c->stream);
      if (e2 != cudaSuccess) return e2;
    }
    // steps lo .. hi-1 again, each keeping its cells' Landau solution, force and streamed h
    // for the reverse step of the same index (the last one's state and next rows are not needed)
    for (int64_t n = lo; n <= hi - 1; ++n) {
      const CUtensorMap *ti = n == lo ? &mck[k] : &msl[(int)((n - lo - 1) & 1)];
      HostStir st = stir_for_step(c, s0 + n);
      if (c->L.nmodes) {
        st.G_cur = gtab((int)(n - lo));
        st.G_next = n == hi - 1 ? w + G.gscratch : gtab((int)(n - lo + 1));
      }
      c->phys.step = s0 + n;
      void *fout = n == hi - 1 ? w + G.scratch : slot((int)((n - lo) & 1));
      CUtensorMap mg_n;  // copied into the launch's parameters
      if (staged_rows) {
        map_error = encode_table_map(c, gtab((int)(n - lo)), &mg_n);
        if (!map_error.empty()) return cudaErrorInvalidValue;
      }
      if ((e2 = dispatch_step_raw(c, ti, fout, s0 + n, st, staged_rows ? &mg_n : nullptr, n > lo,
                                  w + G.macro + G.macro_bytes * (size_t)(n - lo))) != cudaSuccess)
        return e2;
    }
    return cudaSuccess;
  };
  if (one_pass) {
    if ((e = recompute(0, 0, nsteps)) != cudaSuccess) {
      if (!map_error.empty()) return c->fail(RLBM_E_CUDA, map_error);
      return c->cuda_fail(e, "step kernel launch (forward)");
    }
    // the state after the run, B_{N-1}, into a context buffer, as rlbm_step(N) would leave it
    const int dst = c->cur ^ 1;
    if ((e = cudaMemcpyAsync(c->ws + c->L.pop[dst], w + G.scratch, G.state_bytes, cudaMemcpyDeviceToDevice, c->stream)) != cudaSuccess)
      return c->cuda_fail(e, "copy of the final state");
    c->cur = dst;
    c->step = s0 + nsteps;
  }
  int kc = 0;  // kap[kc] holds kappa_{n+1}
  // the last state: objective only (its force terms are multiplied by a zero adjoint)
  a.B = c->ws + c->L.pop[c->cur];
  a.tB = &c->tmap_in[c->cur];
  a.kin = nullptr;
  a.tK = nullptr;
  a.macro = nullptr;  // S_N is no step's input: matched and forced here
  a.kout = w + G.kap[kc];
  a.cj = cj;
  a.G = c->ws + c->L.G[0];
  a.zpart = w + G.zpart;
  if ((e = dispatch_adjoint(c, a)) != cudaSuccess) return c->cuda_fail(e, "adjoint kernel launch");
  for (int k = G.K - 1; k >= 0; --k) {
    const int64_t lo = (int64_t)k * G.seg, hi = std::min<int64_t>(lo + G.seg, nsteps);
    if (!one_pass && (e = recompute(k, lo, hi)) != cudaSuccess) {
      if (!map_error.empty()) return c->fail(RLBM_E_CUDA, map_error);
      return c->cuda_fail(e, "step kernel launch (recompute)");
    }
    for (int64_t n = hi - 1; n >= lo; --n) {
      a.B = ckpt(k);  // (not read: the step's streamed h is in its stored values)
      a.tB = &mck[k];
      a.kin = w + G.kap[kc];
      a.tK = &mkap[kc];
      a.kout = w + G.kap[kc ^ 1];
      a.cj = n >= 1 ? cj : 0.0;
      a.G = gtab((int)(n - lo));
      a.zpart = w + G.zpart + G.zpart_bytes * (size_t)(n - lo);
      a.macro = w + G.macro + G.macro_bytes * (size_t)(n - lo);
      a.chained = n < hi - 1;  // the first reverse step of a segment follows its recomputation
      if ((e = dispatch_adjoint(c, a)) != cudaSuccess) return c->cuda_fail(e, "adjoint kernel launch");
      kc ^= 1;
    }
    mg.nj = (int)(hi - lo);
    mg.n0 = s0 + lo;
    mg.gstep = gstep + (size_t)lo * c->L.nmodes;
    e = c->cfg.precision == RLBM_F64 ? launch_mode_grads_f64(mg, c->stream) : launch_mode_grads_f32(mg, c->stream);
    if (e != cudaSuccess) return c->cuda_fail(e, "mode gradient kernels");
  }
  if ((e = launch_mode_sum(gstep, nsteps, c->L.nmodes, gsig, c->stream)) != cudaSuccess) return c->cuda_fail(e, "mode sum kernel");
  double *out = reinterpret_cast<double *>(w + G.out);
  if ((e = launch_reduce_partials(a.acc, G.nblocks, out, c->stream)) != cudaSuccess) return c->cuda_fail(e, "reduction kernel");
  // the context continues from step s0 + nsteps
  c->phys.step = c->step;
  if ((e = stir_prime(c, c->step)) != cudaSuccess) return c->cuda_fail(e, "stirring set-up kernels");
  double host[4];
  if ((e = cudaMemcpyAsync(host, out, 32, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return c->cuda_fail(e, "copy of the sums");
  if (grad_sigma && c->L.nmodes &&
      (e = cudaMemcpyAsync(grad_sigma, gsig, 8 * (size_t)c->L.nmodes, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return c->cuda_fail(e, "copy of the mode gradient");
  if (rlbm_status s = check_device(c)) return s;
  if (J) *J = host[3];
  if (grad_eta_over_s) *grad_eta_over_s = -host[0] / c->cfg.eta_over_s;
  if (grad_body_force) { grad_body_force[0] = host[1]; grad_body_force[1] = host[2]; }
  return RLBM_OK;
}

}  // extern "C"
