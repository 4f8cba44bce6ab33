// C ABI of liblbm_imb (declared in include/lbm_imb.h): configuration checks,
// layout of the caller's device block, the per-step schedule (captured once
// per ping-pong parity into a CUDA graph), and the synchronising accessors.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "lbm_internal.cuh"

using lbm::View;

namespace lbm {
int batch_max_grid(int dim, int storage, int smem);
int batch_queue_smem(int dim, int storage);
int batch_sm_count();
cudaError_t launch_batch_step(const View* views, int nm, const int* part_off, const int* tile_off,
                              const int* bin_off, const int* tiles_x, int tile_x, int dim, int storage,
                              double rmax, unsigned* bar, int* err, long long spin_limit, int phantom,
                              int grid, int smem, cudaStream_t s);
}  // namespace lbm

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStageMax = 64ull << 20;  // staging for host-side field copies
constexpr int64_t kHealthEvery = 100;      // default steps between health checks

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
  int pitch;
  long long plane;
  int Q;
  size_t esz_f, esz_eps;
  int nb[3];
  double bsz[3];
  double rmax;
  int smem;
  size_t off_f[2], off_own[lbm::kMaxOwners], off_eps[lbm::kMaxOwners];
  size_t off_pos, off_vel, off_omg, off_rad, off_mass, off_inertia, off_ff, off_tf, off_fc;
  size_t off_lo, off_kin, off_binof, off_bincount, off_binslot, off_err, off_red, off_stage;
  size_t off_tab;  // Eq. 6 table (eps_method 1), 0 bytes otherwise
  size_t off_vl_nbr, off_vl_count, off_vl_ref, off_vl_flag;  // Verlet lists (dem_skin > 0)
  size_t off_cov_list, off_cov_count;  // covered-node list (pair storage with particles)
  size_t off_cbuf;                      // covered-node buffer of split form 9 (same)
  long long cbuf_cap;
  size_t stage_bytes;
  size_t total;
};

// particle state the kernels accept: finite velocities and spins, finite
// centres inside the walls (y in [-1/2, ny - 1/2] when wall_y) and in
// [-1/2, n) along periodic axes (the DEM keeps wrapped centres in [0, n);
// any two centres then differ by less than n + 1/2, which one minimum-image
// wrap resolves)
int check_particle_state(int dim, const int ext[3], int wall_y, int64_t n, const double* pos,
                         const double* vel, const double* omega) {
  for (int64_t p = 0; p < n; p++) {
    for (int d = 0; d < 3; d++) {
      if (vel && !isfinite(vel[3 * p + d])) return LBM_IMB_EINVAL;
      if (omega && !isfinite(omega[3 * p + d])) return LBM_IMB_EINVAL;
      if (!pos || d >= dim) continue;
      const double x = pos[3 * p + d], L = (double)ext[d];
      if (!isfinite(x)) return LBM_IMB_EINVAL;
      if (d == 1 && wall_y) {
        if (x < -0.5 || x > L - 0.5) return LBM_IMB_EINVAL;
      } else if (x < -0.5 || x >= L) {
        return LBM_IMB_EINVAL;
      }
    }
  }
  return LBM_IMB_OK;
}

// check_positions = false for the per-slab layouts of a decomposed lattice
// (their configs carry the whole lattice's particles; the whole config was
// checked first)
int validate(const lbm_imb_config* c, bool check_positions = true) {
  if (!c || c->struct_size < sizeof(lbm_imb_config)) return LBM_IMB_EINVAL;
  if (c->dim != 2 && c->dim != 3) return LBM_IMB_EINVAL;
  if (c->nx < 2 || c->ny < 2 || c->nz < 1) return LBM_IMB_EINVAL;
  if (c->dim == 2 && c->nz != 1) return LBM_IMB_EINVAL;
  if (c->ny > 65535 || c->nz > 65535) return LBM_IMB_EUNSUPPORTED;
  if (!(c->tau > 0.5) || !isfinite(c->tau)) return LBM_IMB_EINVAL;
  if (c->storage < 0 || c->storage > 3) return LBM_IMB_EINVAL;
  if (c->wall_y != 0 && c->wall_y != 1) return LBM_IMB_EINVAL;
  if (!(c->rho_fluid > 0.0)) return LBM_IMB_EINVAL;
  if (c->n_particles < 0 || c->n_particles > (1ll << 30)) return LBM_IMB_EINVAL;
  if (c->dem_substeps < 1) return LBM_IMB_EINVAL;
  if (c->eps_method != 0 && c->eps_method != 1) return LBM_IMB_EINVAL;
  if (!(c->dem_skin >= 0.0) || !isfinite(c->dem_skin)) return LBM_IMB_EINVAL;
  if (c->n_particles > 0) {
    if (!c->pos || !c->radius || !c->density) return LBM_IMB_EINVAL;
    if (!(c->k_n >= 0.0) || !(c->restitution > 0.0 && c->restitution <= 1.0)) return LBM_IMB_EINVAL;
    for (int64_t p = 0; p < c->n_particles; p++) {
      if (!(c->radius[p] > 0.0) || !(c->density[p] > 0.0)) return LBM_IMB_EINVAL;
      if (!isfinite(c->radius[p]) || !isfinite(c->density[p])) return LBM_IMB_EINVAL;
    }
    const int ext[3] = {c->nx, c->ny, c->dim == 3 ? c->nz : 1};
    const int st = check_particle_state(c->dim, ext, c->wall_y, c->n_particles, check_positions ? c->pos : nullptr,
                                        c->vel, c->omega);
    if (st) return st;
  }
  return LBM_IMB_OK;
}

// FNV-1a over the configuration's values (not its pointers or padding):
// a checkpoint loads only into a simulation of the same configuration
uint64_t config_hash(const lbm_imb_config* c) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; i++) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  const int32_t ints[9] = {c->dim, c->nx, c->ny, c->dim == 3 ? c->nz : 1, c->wall_y, c->storage,
                           c->dem_substeps, c->eps_method, 0};
  mix(ints, sizeof(ints));
  const double dbl[11] = {c->tau, c->body_force[0], c->body_force[1], c->body_force[2], c->gravity[0],
                          c->gravity[1], c->gravity[2], c->rho_fluid, c->k_n, c->restitution, c->dem_skin};
  mix(dbl, sizeof(dbl));
  const int64_t np = c->n_particles;
  mix(&np, sizeof(np));
  if (np > 0) {
    mix(c->radius, sizeof(double) * (size_t)np);
    mix(c->density, sizeof(double) * (size_t)np);
  }
  return h;
}

int make_layout(const lbm_imb_config* c, Layout* L, bool check_positions = true) {
  int st = validate(c, check_positions);
  if (st) return st;
  const int nz = c->dim == 3 ? c->nz : 1;
  L->Q = c->dim == 2 ? 9 : 19;
  L->pitch = (c->nx + 31) / 32 * 32;
  L->plane = (long long)L->pitch * c->ny * nz;
  if (L->plane >= (1ll << 31)) return LBM_IMB_EUNSUPPORTED;  // 32-bit node offsets
  L->esz_f = lbm::pop_bytes(c->storage);
  L->esz_eps = lbm::fp64_eps(c->storage) ? 8 : 4;
  double rmax = 0.0;
  for (int64_t p = 0; p < c->n_particles; p++) rmax = c->radius[p] > rmax ? c->radius[p] : rmax;
  L->rmax = rmax;
  const int ext[3] = {c->nx, c->ny, nz};
  // Verlet lists need every pair within R_i + R_j + skin in neighbouring bins
  st = lbm::dem_bin_geometry(c->dim, ext, c->wall_y, rmax + 0.5 * c->dem_skin, L->nb, L->bsz);
  if (st) return st;
  L->rmax = rmax;
  L->smem = 0;
  if (c->n_particles > 0) {
    // the exact 3D rasteriser keeps its corner tables in shared memory (R <= 8);
    // the Eq. 6 table form and 2D keep per-axis tables of <= 64 entries
    const double rlim = (c->dim == 3 && c->eps_method == 0) ? 8.0 : 29.0;
    if (rmax > rlim) return LBM_IMB_EUNSUPPORTED;
    if (c->eps_method == 1) {  // one table: one radius, and a cell centre never at the table's r < 0
      for (int64_t p = 0; p < c->n_particles; p++)
        if (c->radius[p] != c->radius[0]) return LBM_IMB_EUNSUPPORTED;
      if (!(c->radius[0] > 1.0)) return LBM_IMB_EUNSUPPORTED;
    }
    L->smem = c->eps_method == 1 ? lbm::eps_table_raster_smem_bytes(c->dim, c->storage, rmax)
                                 : lbm::eps_raster_smem_bytes(c->dim, c->storage, rmax);
    if (L->smem < 0) return LBM_IMB_EUNSUPPORTED;
  }
  const long long nbins = (long long)L->nb[0] * L->nb[1] * L->nb[2];
  const size_t np = (size_t)(c->n_particles > 0 ? c->n_particles : 1);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  for (int k = 0; k < 2; k++) L->off_f[k] = take((size_t)L->Q * L->plane * L->esz_f);
  for (int s = 0; s < lbm::kMaxOwners; s++) L->off_own[s] = take((size_t)L->plane * 4);
  for (int s = 0; s < lbm::kMaxOwners; s++) L->off_eps[s] = take((size_t)L->plane * L->esz_eps);
  L->off_pos = take(np * 24);
  L->off_vel = take(np * 24);
  L->off_omg = take(np * 24);
  L->off_rad = take(np * 8);
  L->off_mass = take(np * 8);
  L->off_inertia = take(np * 8);
  L->off_ff = take(np * 24);
  L->off_tf = take(np * 24);
  L->off_fc = take(np * 24);
  L->off_lo = take(np * 24);
  L->off_kin = take(np * 128);
  L->off_binof = take(np * 4);
  L->off_bincount = take((size_t)nbins * 4);
  L->off_binslot = take((size_t)nbins * lbm::kBinCap * 4);
  L->off_err = take(16);
  L->off_red = take(8 * 8);
  L->off_tab = take(c->eps_method == 1 && c->n_particles > 0 ? (size_t)lbm::eps_table_entries(c->dim) * 4 : 0);
  const bool vl = c->dem_skin > 0.0 && c->n_particles > 0;
  L->off_vl_nbr = take(vl ? np * lbm::kVerletCap * 4 : 0);
  L->off_vl_count = take(vl ? np * 4 : 0);
  L->off_vl_ref = take(vl ? np * 24 : 0);
  L->off_vl_flag = take(16);
  const bool cov = c->storage == LBM_IMB_STORE_DFDEV && c->n_particles > 0;
  L->off_cov_list = take(cov ? (size_t)L->plane * 4 : 0);
  L->off_cov_count = take(16);
  // covered nodes lie in particle boxes of at most (2 rmax + 2)^dim cells
  long long cells = 1;
  for (int d = 0; d < c->dim; d++) cells *= (long long)floor(2.0 * rmax) + 2;
  L->cbuf_cap = cov ? (c->n_particles < L->plane / cells ? c->n_particles * cells : L->plane) : 0;
  L->off_cbuf = take(cov ? (size_t)L->cbuf_cap * ((size_t)(L->Q + 5) * 8 + 20) : 0);
  const size_t dense_row = (size_t)c->nx * 8 * (L->Q > 5 ? L->Q : 5);
  const size_t full = dense_row * (size_t)c->ny * nz;
  L->stage_bytes = full < kStageMax ? full : kStageMax;
  if (L->stage_bytes < dense_row) L->stage_bytes = dense_row;
  L->off_stage = take(L->stage_bytes);
  L->total = o;
  return LBM_IMB_OK;
}

int map_err(int bits) { return lbm::status_of_err_bits(bits); }

}  // namespace

struct lbm_imb {
  View v;  // fsrc/fdst filled per use
  // batch state (is_batch), y-slab decomposition (is_slab), or membership
  // of either (is_member)
  bool is_batch, is_member, is_slab;
  lbm::SlabHalo halo;  // is_slab: halo rows to exchange after every collision
  int nm;
  lbm_imb* members;
  lbm_imb* parent;
  View* d_views[2];  // member views per ping-pong parity (device)
  int *d_part_off, *d_tile_off, *d_bin_off, *d_tiles_x;
  unsigned* d_bar;
  int* d_berr;
  int tile_x, blocks_per_sm, grid, bsmem;
  double rmax_all;
  long long spin_limit;
  int phantom;
  void* f[2];
  int cur;
  cudaStream_t stream;
  int smem;
  cudaGraphExec_t graph[2];
  bool graphs_tried;
  bool graphs_ok;
  int64_t steps;
  int dim, Q, np;
  long long N;
  double* stage;
  size_t stage_bytes;
  int64_t health_every;  // health check every this many steps (0: never)
  uint64_t cfg_hash;     // of the configuration at init (checkpoints)
};

namespace {

View view_of(const lbm_imb* h, int src) {
  View v = h->v;
  v.fsrc = h->f[src];
  v.fdst = h->f[src ^ 1];
  const size_t esz = lbm::pop_bytes(v.storage);
  for (int q = 0; q < 19; q++) {
    const size_t off = q < v.Q ? (size_t)q * (size_t)v.plane * esz : 0;
    v.src_q[q] = static_cast<const unsigned char*>(v.fsrc) + off;
    v.dst_q[q] = static_cast<unsigned char*>(v.fdst) + off;
  }
  return v;
}

// one step of a y-slab decomposition (lbm_imb_slabs_init)
void enqueue_slab_step(lbm_imb* h, int src) {
  for (int k = 0; k < h->nm; k++) {
    lbm_imb* m = h->members + k;
    lbm::launch_eps_clear(view_of(m, src), k == 0, h->stream);  // slab 0 zeroes the force sums
  }
  for (int k = 0; k < h->nm; k++) {
    lbm_imb* m = h->members + k;
    lbm::launch_eps_raster(view_of(m, src), m->smem, h->stream);
  }
  for (int k = 0; k < h->nm; k++) lbm::launch_collide(view_of(h->members + k, src), h->stream);
  lbm::launch_halo_exchange(h->halo, src ^ 1, h->stream);
  lbm::launch_dem(h->v, h->stream);
}

void enqueue_step(lbm_imb* h, int src) {
  if (h->is_slab) {
    enqueue_slab_step(h, src);
    return;
  }
  View v = view_of(h, src);
  lbm::launch_eps_clear(v, true, h->stream);
  lbm::launch_eps_raster(v, h->smem, h->stream);
  lbm::launch_collide(v, h->stream);
  lbm::launch_dem(v, h->stream);
}

// health check of the stored populations and particle state (every member
// of a batch or slab decomposition); sets ERR_NONFINITE, reported by the
// next synchronising call
void enqueue_health(lbm_imb* h) {
  if (h->is_batch || h->is_slab) {
    for (int k = 0; k < h->nm; k++) {
      lbm_imb* m = h->members + k;
      lbm::launch_health(view_of(m, m->cur), m->f[m->cur], h->stream);
    }
    return;
  }
  lbm::launch_health(view_of(h, h->cur), h->f[h->cur], h->stream);
}

void maybe_health(lbm_imb* h) {
  if (h->health_every > 0 && h->steps % h->health_every == 0) enqueue_health(h);
}

void try_capture(lbm_imb* h) {
  h->graphs_tried = true;
  h->graphs_ok = false;
  if (h->stream == nullptr) return;  // the legacy stream cannot be captured
  for (int k = 0; k < 2; k++) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    enqueue_step(h, k);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess || g == nullptr) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      if (k == 1) cudaGraphExecDestroy(h->graph[0]);
      return;
    }
    e = cudaGraphInstantiate(&h->graph[k], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (k == 1) cudaGraphExecDestroy(h->graph[0]);
      return;
    }
  }
  h->graphs_ok = true;
}

int check_cuda(cudaError_t e) { return e == cudaSuccess ? LBM_IMB_OK : LBM_IMB_ECUDA; }

int read_err(lbm_imb* h) {
  int bits = 0;
  if (cudaMemcpyAsync(&bits, h->v.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
    return LBM_IMB_ECUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LBM_IMB_ECUDA;
  if (bits) {
    cudaMemsetAsync(h->v.err, 0, sizeof(int), h->stream);
    cudaStreamSynchronize(h->stream);
  }
  return map_err(bits);
}

long long rows_per_chunk(const lbm_imb* h, int comps) {
  const long long per_row = (long long)h->v.nx * 8 * comps;
  long long r = (long long)(h->stage_bytes / per_row);
  return r < 1 ? 1 : r;
}

}  // namespace

// lay out one simulation in its device block and initialise it
// a y slab of a decomposed lattice (see View::y0); null for a whole lattice
struct SlabGeom {
  int y0, ny_c, ygo, ny_glob, wall_lo, wall_hi, wall_y;
};

static int setup_handle(lbm_imb* h, const lbm_imb_config* c, void* dev_buf, const Layout& L,
                        cudaStream_t stream, const SlabGeom* sg = nullptr) {
  h->stream = stream;
  unsigned char* base = static_cast<unsigned char*>(dev_buf);
  const int nz = c->dim == 3 ? c->nz : 1;
  const int np = (int)c->n_particles;
  View& v = h->v;
  memset(&v, 0, sizeof(v));
  v.dim = c->dim;
  v.Q = L.Q;
  v.nx = c->nx;
  v.ny = c->ny;
  v.nz = nz;
  v.pitch = L.pitch;
  v.plane = L.plane;
  v.wall_y = c->wall_y;
  v.storage = c->storage;
  v.y0 = 0;
  v.ny_c = c->ny;
  v.ygo = 0;
  v.ny_glob = c->ny;
  v.wall_lo = v.wall_hi = c->wall_y;
  if (sg) {
    v.y0 = sg->y0;
    v.ny_c = sg->ny_c;
    v.ygo = sg->ygo;
    v.ny_glob = sg->ny_glob;
    v.wall_lo = sg->wall_lo;
    v.wall_hi = sg->wall_hi;
    v.wall_y = sg->wall_y;
  }
  for (int s = 0; s < lbm::kMaxOwners; s++) {
    v.own[s] = reinterpret_cast<int*>(base + L.off_own[s]);
    v.eps[s] = base + L.off_eps[s];
  }
  v.np = np;
  v.pos = reinterpret_cast<double*>(base + L.off_pos);
  v.vel = reinterpret_cast<double*>(base + L.off_vel);
  v.omg = reinterpret_cast<double*>(base + L.off_omg);
  v.rad = reinterpret_cast<double*>(base + L.off_rad);
  v.mass = reinterpret_cast<double*>(base + L.off_mass);
  v.inertia = reinterpret_cast<double*>(base + L.off_inertia);
  v.ff = reinterpret_cast<double*>(base + L.off_ff);
  v.tf = reinterpret_cast<double*>(base + L.off_tf);
  v.fc = reinterpret_cast<double*>(base + L.off_fc);
  v.lo = reinterpret_cast<int*>(base + L.off_lo);
  v.kin = reinterpret_cast<float*>(base + L.off_kin);
  v.bin_of = reinterpret_cast<int*>(base + L.off_binof);
  for (int d = 0; d < 3; d++) {
    v.nb[d] = L.nb[d];
    v.bsz[d] = L.bsz[d];
  }
  v.bin_count = reinterpret_cast<int*>(base + L.off_bincount);
  v.bin_slot = reinterpret_cast<int*>(base + L.off_binslot);
  v.rmax_bins = L.rmax;
  v.tau = c->tau;
  v.omega = 1.0 / c->tau;
  for (int d = 0; d < 3; d++) {
    v.gf[d] = (d < c->dim) ? c->body_force[d] : 0.0;
    v.gs[d] = (d < c->dim) ? c->gravity[d] : 0.0;
  }
  v.rho0 = c->rho_fluid;
  v.kn = c->k_n;
  const double le = log(c->restitution);
  v.ln_e = le;
  v.dem_den = M_PI * M_PI + le * le;
  v.substeps = c->dem_substeps;
  for (int q = 0; q < 19; q++) {
    double cg = 0.0, w = 0.0;
    if (q < L.Q) {
      if (c->dim == 2) {
        cg = lbm::D2Q9::c(q, 0) * v.gf[0] + lbm::D2Q9::c(q, 1) * v.gf[1];
        w = lbm::D2Q9::w(q);
      } else {
        cg = lbm::D3Q19::c(q, 0) * v.gf[0] + lbm::D3Q19::c(q, 1) * v.gf[1] + lbm::D3Q19::c(q, 2) * v.gf[2];
        w = lbm::D3Q19::w(q);
      }
    }
    v.fq[q] = 3.0 * w * cg;
    v.fq_f[q] = (float)v.fq[q];
    v.cg3[q] = 3.0 * cg;
    v.cg3_f[q] = (float)v.cg3[q];
  }
  v.omc = 1.0 - v.omega;
  v.omc_f = (float)v.omc;
  v.tau_f = (float)v.tau;
  v.omega_f = (float)v.omega;
  v.rho0_f = (float)v.rho0;
  auto split = [](double d, float* p) {  // high and low FP32 parts
    p[0] = (float)d;
    p[1] = (float)(d - (double)p[0]);
  };
  split(v.omc, v.omc_df);
  split(v.tau, v.tau_df);
  split(v.omega, v.omega_df);
  split(v.rho0, v.rho0_df);
  for (int q = 0; q < 19; q++) {
    split(v.fq[q], v.fq_df[q]);
    split(v.cg3[q], v.cg3_df[q]);
  }
  v.err = reinterpret_cast<int*>(base + L.off_err);
  v.red = reinterpret_cast<double*>(base + L.off_red);
  v.eps_method = np > 0 ? c->eps_method : 0;
  v.dem_skin = np > 0 ? c->dem_skin : 0.0;
  v.vl_nbr = reinterpret_cast<int*>(base + L.off_vl_nbr);
  v.vl_count = reinterpret_cast<int*>(base + L.off_vl_count);
  v.vl_ref = reinterpret_cast<double*>(base + L.off_vl_ref);
  v.vl_flag = reinterpret_cast<int*>(base + L.off_vl_flag);
  v.vl_builds = reinterpret_cast<long long*>(base + L.off_vl_flag + 8);
  v.eps_tab = reinterpret_cast<const float*>(base + L.off_tab);
  const bool cov = c->storage == LBM_IMB_STORE_DFDEV && np > 0;
  v.cov_list = cov ? reinterpret_cast<int*>(base + L.off_cov_list) : nullptr;
  v.cov_count = cov ? reinterpret_cast<int*>(base + L.off_cov_count) : nullptr;
  v.cbuf = cov ? reinterpret_cast<float2*>(base + L.off_cbuf) : nullptr;
  v.cbuf_cap = cov ? L.cbuf_cap : 0;
  v.tab_lo_r = v.tab_h_r = v.tab_h_s = v.tab_h_t = 0.f;
  if (v.eps_method == 1)
    lbm::eps_table_geometry(c->dim, c->radius[0], &v.tab_lo_r, &v.tab_h_r, &v.tab_h_s, &v.tab_h_t);
  h->f[0] = base + L.off_f[0];
  h->f[1] = base + L.off_f[1];
  h->cur = 0;
  h->smem = L.smem;
  h->dim = c->dim;
  h->Q = L.Q;
  h->np = np;
  h->N = (long long)c->nx * c->ny * nz;
  h->stage = reinterpret_cast<double*>(base + L.off_stage);
  h->stage_bytes = L.stage_bytes;
  h->health_every = kHealthEvery;
  h->cfg_hash = config_hash(c);

  // particle state on the host first (derived masses as in the method)
  int st = LBM_IMB_OK;
  if (np > 0) {
    double* hbuf = (double*)malloc(sizeof(double) * (size_t)np * 15);
    if (!hbuf) return LBM_IMB_ENOMEM;
    double *hp = hbuf, *hv = hbuf + 3 * np, *hw = hbuf + 6 * np, *hr = hbuf + 9 * np,
           *hm = hbuf + 10 * np, *hi = hbuf + 11 * np;
    for (int p = 0; p < np; p++) {
      for (int d = 0; d < 3; d++) {
        hp[3 * p + d] = c->pos[3 * p + d];
        hv[3 * p + d] = c->vel ? c->vel[3 * p + d] : 0.0;
        hw[3 * p + d] = c->omega ? c->omega[3 * p + d] : 0.0;
      }
      if (c->dim == 2) {
        hp[3 * p + 2] = 0.0;
        hv[3 * p + 2] = 0.0;
        hw[3 * p + 0] = 0.0;
        hw[3 * p + 1] = 0.0;
      }
      const double R = c->radius[p];
      hr[p] = R;
      if (c->dim == 2) {
        hm[p] = c->density[p] * M_PI * R * R;
        hi[p] = 0.5 * hm[p] * R * R;
      } else {
        hm[p] = c->density[p] * (4.0 / 3.0) * M_PI * R * R * R;
        hi[p] = 0.4 * hm[p] * R * R;
      }
    }
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpyAsync(v.pos, hp, 24ull * np, cudaMemcpyHostToDevice, h->stream);
    e = e ? e : cudaMemcpyAsync(v.vel, hv, 24ull * np, cudaMemcpyHostToDevice, h->stream);
    e = e ? e : cudaMemcpyAsync(v.omg, hw, 24ull * np, cudaMemcpyHostToDevice, h->stream);
    e = e ? e : cudaMemcpyAsync(v.rad, hr, 8ull * np, cudaMemcpyHostToDevice, h->stream);
    e = e ? e : cudaMemcpyAsync(v.mass, hm, 8ull * np, cudaMemcpyHostToDevice, h->stream);
    e = e ? e : cudaMemcpyAsync(v.inertia, hi, 8ull * np, cudaMemcpyHostToDevice, h->stream);
    e = e ? e : cudaMemsetAsync(v.ff, 0, 24ull * np, h->stream);
    e = e ? e : cudaMemsetAsync(v.tf, 0, 24ull * np, h->stream);
    e = e ? e : cudaMemsetAsync(v.fc, 0, 24ull * np, h->stream);
    e = e ? e : cudaStreamSynchronize(h->stream);
    free(hbuf);
    if (e != cudaSuccess) st = LBM_IMB_ECUDA;
    if (!st && L.smem > 0 && lbm::eps_raster_set_attrs(L.smem) != 0) st = LBM_IMB_ECUDA;
  }
  if (!st) {
    cudaError_t e = cudaMemsetAsync(v.err, 0, 16, h->stream);
    if (e == cudaSuccess && v.cov_count) e = cudaMemsetAsync(v.cov_count, 0, 16, h->stream);
    for (int s = 0; s < lbm::kMaxOwners && e == cudaSuccess; s++)
      e = cudaMemsetAsync(v.own[s], 0xff, (size_t)L.plane * 4, h->stream);
    if (e == cudaSuccess && v.eps_method == 1)
      e = lbm::launch_eps_table_build(c->dim, c->radius[0], const_cast<float*>(v.eps_tab), h->stream);
    if (e == cudaSuccess) {  // Verlet: first pass builds; no builds yet
      const long long flag_builds[2] = {1, 0};
      e = cudaMemcpyAsync(v.vl_flag, flag_builds, 16, cudaMemcpyHostToDevice, h->stream);
    }
    if (e == cudaSuccess) {
      View v0 = view_of(h, 0);
      lbm::launch_init_equilibrium(v0, h->f[0], h->stream);
      lbm::launch_init_equilibrium(v0, h->f[1], h->stream);
      lbm::launch_eps_raster(v0, h->smem, h->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = LBM_IMB_ECUDA;
  }
  if (!st) st = read_err(h);
  return st;
}

static void lbm_imb_destroy_member_graphs(lbm_imb* m) {
  if (m->graphs_ok) {
    cudaGraphExecDestroy(m->graph[0]);
    cudaGraphExecDestroy(m->graph[1]);
  }
  m->graphs_ok = false;
}

// ---- batch plumbing ----
struct BatchLayout {
  size_t off_views[2], off_part, off_tile, off_bin, off_tx, off_bar, off_berr, header;
  size_t member_off[256];
  Layout member[256];
  size_t total;
};

static int batch_layout(const lbm_imb_config* cfgs, int n, BatchLayout* B) {
  if (!cfgs || n < 1 || n > 256) return LBM_IMB_EINVAL;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  B->off_views[0] = take(sizeof(View) * n);
  B->off_views[1] = take(sizeof(View) * n);
  B->off_part = take(4 * (n + 1));
  B->off_tile = take(4 * (n + 1));
  B->off_bin = take(4 * (n + 1));
  B->off_tx = take(4 * n);
  B->off_bar = take(16);
  B->off_berr = take(16);
  B->header = o;
  for (int i = 0; i < n; i++) {
    const lbm_imb_config* c = cfgs + i;
    int st = make_layout(c, &B->member[i]);
    if (st) return st;
    if (c->dim != cfgs[0].dim || c->storage != cfgs[0].storage) return LBM_IMB_EINVAL;
    if (c->dem_substeps != 1) return LBM_IMB_EUNSUPPORTED;
    if (c->dem_skin != 0.0) return LBM_IMB_EUNSUPPORTED;
    if (c->storage == LBM_IMB_STORE_DFDEV) return LBM_IMB_EUNSUPPORTED;
    B->member_off[i] = take(B->member[i].total);
  }
  B->total = o;
  return LBM_IMB_OK;
}

static void batch_drop_graphs(lbm_imb* h) {
  if (h->graphs_ok) {
    cudaGraphExecDestroy(h->graph[0]);
    cudaGraphExecDestroy(h->graph[1]);
  }
  h->graphs_ok = false;
  h->graphs_tried = false;
}

// member views for both parities and the work-list prefixes for tile_x
static int batch_upload(lbm_imb* h) {
  const int n = h->nm;
  View* hv = (View*)malloc(sizeof(View) * n * 2);
  int* hi = (int*)malloc(sizeof(int) * (4 * (n + 1)));
  if (!hv || !hi) {
    free(hv);
    free(hi);
    return LBM_IMB_ENOMEM;
  }
  int *part = hi, *tile = hi + (n + 1), *bin = hi + 2 * (n + 1), *tx = hi + 3 * (n + 1);
  part[0] = tile[0] = bin[0] = 0;
  const int ty = 128 / h->tile_x;
  for (int i = 0; i < n; i++) {
    lbm_imb* m = h->members + i;
    for (int k = 0; k < 2; k++) hv[k * n + i] = view_of(m, k);
    const int rows = m->v.ny * m->v.nz;
    tx[i] = (m->v.nx + h->tile_x - 1) / h->tile_x;
    part[i + 1] = part[i] + m->np;
    tile[i + 1] = tile[i] + tx[i] * ((rows + ty - 1) / ty);
    bin[i + 1] = bin[i] + (m->np > 0 ? m->v.nb[0] * m->v.nb[1] * m->v.nb[2] : 0);
  }
  cudaError_t e = cudaMemcpyAsync(h->d_views[0], hv, sizeof(View) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_views[1], hv + n, sizeof(View) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_part_off, part, 4 * (n + 1), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_tile_off, tile, 4 * (n + 1), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_bin_off, bin, 4 * (n + 1), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_tiles_x, tx, 4 * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_bar, 0, 16, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_berr, 0, 16, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free(hv);
  free(hi);
  return e == cudaSuccess ? LBM_IMB_OK : LBM_IMB_ECUDA;
}

static int batch_configure(lbm_imb* h, int tile_x, int blocks_per_sm) {
  if (tile_x == 0) tile_x = 128;
  if (tile_x != 32 && tile_x != 64 && tile_x != 128) return LBM_IMB_EINVAL;
  if (blocks_per_sm < 0) return LBM_IMB_EINVAL;
  const int max_grid = lbm::batch_max_grid(h->dim, h->v.storage, h->bsmem);
  if (max_grid <= 0) return LBM_IMB_ECUDA;
  const int sms = lbm::batch_sm_count();
  int grid = blocks_per_sm > 0 ? blocks_per_sm * sms : max_grid;
  if (grid > max_grid) grid = max_grid;
  if (grid < 1) return LBM_IMB_EUNSUPPORTED;
  batch_drop_graphs(h);
  h->tile_x = tile_x;
  h->blocks_per_sm = blocks_per_sm;
  h->grid = grid;
  return batch_upload(h);
}

static cudaError_t batch_enqueue(lbm_imb* h, int parity) {
  return lbm::launch_batch_step(h->d_views[parity], h->nm, h->d_part_off, h->d_tile_off, h->d_bin_off,
                                h->d_tiles_x, h->tile_x, h->dim, h->v.storage, h->rmax_all, h->d_bar,
                                h->d_berr, h->spin_limit, h->phantom, h->grid, h->bsmem, h->stream);
}

static void batch_try_capture(lbm_imb* h) {
  h->graphs_tried = true;
  h->graphs_ok = false;
  if (h->stream == nullptr) return;
  for (int k = 0; k < 2; k++) {
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      if (k == 1) cudaGraphExecDestroy(h->graph[0]);
      return;
    }
    cudaError_t e1 = batch_enqueue(h, k);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e1 != cudaSuccess || e != cudaSuccess || g == nullptr ||
        cudaGraphInstantiate(&h->graph[k], g, 0) != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      if (k == 1) cudaGraphExecDestroy(h->graph[0]);
      return;
    }
    cudaGraphDestroy(g);
  }
  h->graphs_ok = true;
}

static int batch_read_err(lbm_imb* h) {
  int st = LBM_IMB_OK;
  int bits = 0;
  if (cudaMemcpyAsync(&bits, h->d_berr, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LBM_IMB_ECUDA;
  if (bits) {
    // a timed-out barrier leaves its counters mid-way: reset them
    cudaMemsetAsync(h->d_bar, 0, 16, h->stream);
    cudaMemsetAsync(h->d_berr, 0, 16, h->stream);
    cudaStreamSynchronize(h->stream);
    st = map_err(bits);
  }
  for (int i = 0; i < h->nm; i++) {
    const int s2 = read_err(h->members + i);
    if (!st) st = s2;
  }
  return st;
}

extern "C" {

size_t lbm_imb_batch_required_bytes(const lbm_imb_config* cfgs, int n) {
  BatchLayout* B = (BatchLayout*)malloc(sizeof(BatchLayout));
  if (!B) return 0;
  size_t t = batch_layout(cfgs, n, B) == LBM_IMB_OK ? B->total : 0;
  free(B);
  return t;
}

int lbm_imb_batch_init(const lbm_imb_config* cfgs, int n, int tile_x, int blocks_per_sm, void* dev_buf,
                       size_t bytes, void* cuda_stream, lbm_imb_t** out) {
  if (!out) return LBM_IMB_EINVAL;
  BatchLayout* B = (BatchLayout*)malloc(sizeof(BatchLayout));
  if (!B) return LBM_IMB_ENOMEM;
  int st = batch_layout(cfgs, n, B);  // the configurations' own status first
  if (!st && (!dev_buf || ((uintptr_t)dev_buf) % kAlign)) st = LBM_IMB_EINVAL;
  if (!st && bytes < B->total) st = LBM_IMB_ENOMEM;
  lbm_imb* h = nullptr;
  if (!st) {
    h = new (std::nothrow) lbm_imb();
    if (!h) st = LBM_IMB_ENOMEM;
  }
  if (!st) {
    h->members = new (std::nothrow) lbm_imb[n]();
    if (!h->members) st = LBM_IMB_ENOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(dev_buf);
  if (!st) {
    h->is_batch = true;
    h->nm = n;
    h->health_every = kHealthEvery;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->dim = cfgs[0].dim;
    h->v.storage = cfgs[0].storage;
    h->d_views[0] = reinterpret_cast<View*>(base + B->off_views[0]);
    h->d_views[1] = reinterpret_cast<View*>(base + B->off_views[1]);
    h->d_part_off = reinterpret_cast<int*>(base + B->off_part);
    h->d_tile_off = reinterpret_cast<int*>(base + B->off_tile);
    h->d_bin_off = reinterpret_cast<int*>(base + B->off_bin);
    h->d_tiles_x = reinterpret_cast<int*>(base + B->off_tx);
    h->d_bar = reinterpret_cast<unsigned*>(base + B->off_bar);
    h->d_berr = reinterpret_cast<int*>(base + B->off_berr);
    h->spin_limit = 1ll << 25;
    h->rmax_all = 0.0;
    for (int i = 0; i < n && !st; i++) {
      lbm_imb* m = h->members + i;
      st = setup_handle(m, cfgs + i, base + B->member_off[i], B->member[i], h->stream);
      m->is_member = true;
      m->parent = h;
      if (B->member[i].rmax > h->rmax_all) h->rmax_all = B->member[i].rmax;
    }
  }
  if (!st) {
    h->bsmem = 0;
    if (h->rmax_all > 0.0) {
      h->bsmem = lbm::eps_raster_smem_bytes(h->dim, h->v.storage, h->rmax_all);
      if (h->bsmem < 0) st = LBM_IMB_EUNSUPPORTED;
    }
    // the collision phase reuses the dynamic shared memory for its queues
    const int qb = lbm::batch_queue_smem(h->dim, h->v.storage);
    if (!st && h->bsmem < qb) h->bsmem = qb;
  }
  if (!st) st = batch_configure(h, tile_x, blocks_per_sm);
  free(B);
  if (st) {
    if (h) {
      delete[] h->members;
      delete h;
    }
    return st;
  }
  *out = h;
  return LBM_IMB_OK;
}

// ---------------------------------------------------------------------------
// y slabs: one lattice decomposed along y on one device.  Slab s holds
// ny_s computed rows (ny split as evenly as possible, the first ny % ns
// slabs one row more) between two halo rows; after every collision a halo
// kernel copies the boundary rows of the post-collision populations into
// the neighbours' halos (across the ends too when y is periodic), the
// exchange a multi-GPU run makes over NVLink.  The particles, their force
// sums and the DEM are shared: every slab rasterises the particles into its
// own rows and adds its Eq. 3 sums to the same FP64 accumulators; the DEM
// runs once per step on the whole domain.
// ---------------------------------------------------------------------------
struct SlabLayout {
  int ns, ny_s[16];
  Layout L[16];
  size_t off[16];
  size_t off_bincount, off_binslot;
  int nb[3];
  double bsz[3];
  size_t total;
};

static void slab_config(const lbm_imb_config* c, int ny_s, lbm_imb_config* out) {
  *out = *c;
  out->ny = ny_s + 2;
  out->wall_y = 1;  // layout only: the slab's walls and halos come from its SlabGeom
}

static int slab_layout(const lbm_imb_config* c, int ns, SlabLayout* S) {
  if (!c || ns < 2 || ns > 16) return LBM_IMB_EINVAL;
  Layout G;
  int st = make_layout(c, &G);
  if (st) return st;
  if (c->dem_skin != 0.0) return LBM_IMB_EUNSUPPORTED;
  S->ns = ns;
  const int base = c->ny / ns, rem = c->ny % ns;
  size_t o = 0;
  for (int k = 0; k < ns; k++) {
    S->ny_s[k] = base + (k < rem ? 1 : 0);
    if (S->ny_s[k] < 2) return LBM_IMB_EUNSUPPORTED;
    lbm_imb_config cs;
    slab_config(c, S->ny_s[k], &cs);
    st = make_layout(&cs, &S->L[k], false);
    if (st) return st;
    S->off[k] = o;
    o = align_up(o + S->L[k].total);
  }
  for (int d = 0; d < 3; d++) {
    S->nb[d] = G.nb[d];
    S->bsz[d] = G.bsz[d];
  }
  const size_t nbins = (size_t)G.nb[0] * G.nb[1] * G.nb[2];
  S->off_bincount = o;
  o = align_up(o + nbins * 4);
  S->off_binslot = o;
  o = align_up(o + nbins * lbm::kBinCap * 4);
  S->total = o;
  return LBM_IMB_OK;
}

size_t lbm_imb_slabs_required_bytes(const lbm_imb_config* cfg, int nslabs) {
  SlabLayout* S = (SlabLayout*)malloc(sizeof(SlabLayout));
  if (!S) return 0;
  const size_t t = slab_layout(cfg, nslabs, S) == LBM_IMB_OK ? S->total : 0;
  free(S);
  return t;
}

int lbm_imb_slabs_init(const lbm_imb_config* c, int nslabs, void* dev_buf, size_t bytes, void* cuda_stream,
                       lbm_imb_t** out) {
  if (!out) return LBM_IMB_EINVAL;
  SlabLayout* S = (SlabLayout*)malloc(sizeof(SlabLayout));
  if (!S) return LBM_IMB_ENOMEM;
  int st = slab_layout(c, nslabs, S);  // the configuration's own status first
  if (!st && (!dev_buf || ((uintptr_t)dev_buf) % kAlign)) st = LBM_IMB_EINVAL;
  if (!st && bytes < S->total) st = LBM_IMB_ENOMEM;
  lbm_imb* h = nullptr;
  if (!st) {
    h = new (std::nothrow) lbm_imb();
    if (!h) st = LBM_IMB_ENOMEM;
  }
  if (!st) {
    h->members = new (std::nothrow) lbm_imb[nslabs]();
    if (!h->members) st = LBM_IMB_ENOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(dev_buf);
  if (!st) {
    h->is_slab = true;
    h->nm = nslabs;
    h->health_every = kHealthEvery;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    int y_start = 0;
    for (int k = 0; k < nslabs && !st; k++) {
      lbm_imb* m = h->members + k;
      lbm_imb_config cs;
      slab_config(c, S->ny_s[k], &cs);
      SlabGeom g;
      g.y0 = 1;
      g.ny_c = S->ny_s[k];
      g.ygo = y_start - 1;
      g.ny_glob = c->ny;
      g.wall_lo = c->wall_y && k == 0;
      g.wall_hi = c->wall_y && k == nslabs - 1;
      g.wall_y = c->wall_y;
      st = setup_handle(m, &cs, base + S->off[k], S->L[k], h->stream, &g);
      m->is_member = true;
      m->parent = h;
      y_start += S->ny_s[k];
    }
  }
  if (!st) {
    // one particle state for every slab (slab 0's arrays), one error word
    const View& p0 = h->members[0].v;
    for (int k = 1; k < nslabs; k++) {
      View& vk = h->members[k].v;
      vk.pos = p0.pos; vk.vel = p0.vel; vk.omg = p0.omg; vk.rad = p0.rad;
      vk.mass = p0.mass; vk.inertia = p0.inertia; vk.ff = p0.ff; vk.tf = p0.tf; vk.fc = p0.fc;
      vk.lo = p0.lo; vk.kin = p0.kin; vk.bin_of = p0.bin_of; vk.err = p0.err; vk.red = p0.red;
    }
    // the handle's own view: the whole domain, for the DEM and the particle calls
    View& v = h->v;
    v = p0;
    v.ny = c->ny;
    v.y0 = 0;
    v.ny_c = c->ny;
    v.ygo = 0;
    v.ny_glob = c->ny;
    v.wall_y = v.wall_lo = v.wall_hi = c->wall_y;
    for (int d = 0; d < 3; d++) {
      v.nb[d] = S->nb[d];
      v.bsz[d] = S->bsz[d];
    }
    v.bin_count = reinterpret_cast<int*>(base + S->off_bincount);
    v.bin_slot = reinterpret_cast<int*>(base + S->off_binslot);
    h->dim = c->dim;
    h->Q = h->members[0].Q;
    h->np = h->members[0].np;
    h->N = (long long)c->nx * c->ny * (c->dim == 3 ? c->nz : 1);
    h->smem = h->members[0].smem;
    lbm::SlabHalo& hb = h->halo;
    memset(&hb, 0, sizeof(hb));
    const size_t esz = lbm::pop_bytes(c->storage);
    for (int k = 0; k < nslabs; k++) {
      hb.f[0][k] = static_cast<unsigned char*>(h->members[k].f[0]);
      hb.f[1][k] = static_cast<unsigned char*>(h->members[k].f[1]);
      hb.ny[k] = S->ny_s[k] + 2;
      hb.plane_bytes[k] = (long long)S->L[k].plane * (long long)esz;
    }
    hb.ns = nslabs;
    hb.periodic = !c->wall_y;
    hb.row_bytes = (int)(S->L[0].pitch * esz);
    hb.nz = c->dim == 3 ? c->nz : 1;
    int nup = 0, ndn = 0;
    for (int q = 0; q < h->members[0].Q; q++) {
      const int cy = c->dim == 2 ? lbm::D2Q9::c(q, 1) : lbm::D3Q19::c(q, 1);
      if (cy == 1) hb.qdir[0][nup++] = q;
      if (cy == -1) hb.qdir[1][ndn++] = q;
    }
    hb.nq = nup;  // == ndn: the directions come in opposite pairs
    // the halos of the initial state
    if (lbm::launch_halo_exchange(hb, 0, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      st = LBM_IMB_ECUDA;
  }
  free(S);
  if (st) {
    if (h) {
      delete[] h->members;
      delete h;
    }
    return st;
  }
  *out = h;
  return LBM_IMB_OK;
}

int lbm_imb_slab_member(lbm_imb_t* h, int i, lbm_imb_t** member) {
  if (!h || !member || !h->is_slab || i < 0 || i >= h->nm) return LBM_IMB_EINVAL;
  *member = h->members + i;
  return LBM_IMB_OK;
}

int lbm_imb_batch_member(lbm_imb_t* h, int i, lbm_imb_t** member) {
  if (!h || !member || !h->is_batch || i < 0 || i >= h->nm) return LBM_IMB_EINVAL;
  *member = h->members + i;
  return LBM_IMB_OK;
}

int lbm_imb_batch_size(lbm_imb_t* h, int* n) {
  if (!h || !n) return LBM_IMB_EINVAL;
  *n = h->is_batch ? h->nm : 1;
  return LBM_IMB_OK;
}

int lbm_imb_batch_set_launch(lbm_imb_t* h, int tile_x, int blocks_per_sm) {
  if (!h || !h->is_batch) return LBM_IMB_EINVAL;
  return batch_configure(h, tile_x, blocks_per_sm);
}

int lbm_imb_batch_get_launch(lbm_imb_t* h, int* tile_x, int* grid) {
  if (!h || !h->is_batch) return LBM_IMB_EINVAL;
  if (tile_x) *tile_x = h->tile_x;
  if (grid) *grid = h->grid;
  return LBM_IMB_OK;
}

int lbm_imb_batch_set_barrier_test(lbm_imb_t* h, int64_t spin_limit, int phantom_arrivals) {
  if (!h || !h->is_batch || spin_limit < 1 || phantom_arrivals < 0) return LBM_IMB_EINVAL;
  batch_drop_graphs(h);
  h->spin_limit = spin_limit;
  h->phantom = phantom_arrivals;
  return LBM_IMB_OK;
}

}  // extern "C"

extern "C" {

size_t lbm_imb_required_bytes(const lbm_imb_config* cfg) {
  Layout L;
  if (make_layout(cfg, &L) != LBM_IMB_OK) return 0;
  return L.total;
}

int lbm_imb_init(const lbm_imb_config* c, void* dev_buf, size_t bytes, void* cuda_stream,
                 lbm_imb_t** out) {
  if (!out) return LBM_IMB_EINVAL;
  Layout L;
  int st = make_layout(c, &L);  // the configuration's own status first
  if (st) return st;
  if (!dev_buf) return LBM_IMB_EINVAL;
  if (bytes < L.total) return LBM_IMB_ENOMEM;
  if (((uintptr_t)dev_buf) % kAlign) return LBM_IMB_EINVAL;
  lbm_imb* h = new (std::nothrow) lbm_imb();
  if (!h) return LBM_IMB_ENOMEM;
  st = setup_handle(h, c, dev_buf, L, static_cast<cudaStream_t>(cuda_stream));
  if (st) {
    delete h;
    return st;
  }
  *out = h;
  return LBM_IMB_OK;
}

int lbm_imb_step(lbm_imb_t* h, int64_t n) {
  if (!h || n < 0 || h->is_member) return LBM_IMB_EINVAL;
  if (n == 0) return LBM_IMB_OK;
  if (h->is_batch) {
    if (!h->graphs_tried) batch_try_capture(h);
    for (int64_t i = 0; i < n; i++) {
      cudaError_t e = h->graphs_ok ? cudaGraphLaunch(h->graph[h->cur], h->stream) : batch_enqueue(h, h->cur);
      if (e != cudaSuccess) return LBM_IMB_ECUDA;
      h->cur ^= 1;
      h->steps++;
      for (int k = 0; k < h->nm; k++) {
        h->members[k].cur = h->cur;
        h->members[k].steps = h->steps;
      }
      maybe_health(h);
    }
    return check_cuda(cudaGetLastError());
  }
  if (!h->graphs_tried) try_capture(h);
  for (int64_t i = 0; i < n; i++) {
    if (h->graphs_ok) {
      if (cudaGraphLaunch(h->graph[h->cur], h->stream) != cudaSuccess) return LBM_IMB_ECUDA;
    } else {
      enqueue_step(h, h->cur);
    }
    h->cur ^= 1;
    h->steps++;
    for (int k = 0; h->is_slab && k < h->nm; k++) {
      h->members[k].cur = h->cur;
      h->members[k].steps = h->steps;
    }
    maybe_health(h);
  }
  return check_cuda(cudaGetLastError());
}

int lbm_imb_step_profiled(lbm_imb_t* h, int64_t n, double* kernel_ms, double* total_ms) {
  if (h && h->is_slab) return LBM_IMB_EUNSUPPORTED;
  if (!h || n < 1 || n > 4096 || !kernel_ms || !total_ms || h->is_member) return LBM_IMB_EINVAL;
  if (h->is_batch) {
    // one persistent launch per step: its time goes to the collide slot
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LBM_IMB_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      return LBM_IMB_ECUDA;
    }
    cudaEventRecord(e0, h->stream);
    int st = lbm_imb_step(h, n);
    cudaEventRecord(e1, h->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (e != cudaSuccess) return LBM_IMB_ECUDA;
    for (int k = 0; k < LBM_IMB_NUM_KERNELS; k++) kernel_ms[k] = 0.0;
    kernel_ms[LBM_IMB_K_COLLIDE] = ms;
    *total_ms = ms;
    return batch_read_err(h);
  }
  const int K = LBM_IMB_NUM_KERNELS;
  const size_t ne = (size_t)n * (K + 1);
  cudaEvent_t* ev = (cudaEvent_t*)calloc(ne, sizeof(cudaEvent_t));
  if (!ev) return LBM_IMB_ENOMEM;
  cudaError_t e = cudaSuccess;
  size_t made = 0;
  for (; made < ne && e == cudaSuccess; made++) e = cudaEventCreate(&ev[made]);
  for (int64_t i = 0; i < n && e == cudaSuccess; i++) {
    View v = view_of(h, h->cur);
    cudaEvent_t* s = ev + i * (K + 1);
    cudaEventRecord(s[0], h->stream);
    lbm::launch_eps_clear(v, true, h->stream);
    cudaEventRecord(s[1], h->stream);
    lbm::launch_eps_raster(v, h->smem, h->stream);
    cudaEventRecord(s[2], h->stream);
    lbm::launch_collide(v, h->stream);
    cudaEventRecord(s[3], h->stream);
    lbm::launch_dem(v, h->stream);
    e = cudaEventRecord(s[4], h->stream);
    h->cur ^= 1;
    h->steps++;
    maybe_health(h);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) {
    for (int k = 0; k < K; k++) kernel_ms[k] = 0.0;
    for (int64_t i = 0; i < n; i++) {
      cudaEvent_t* s = ev + i * (K + 1);
      for (int k = 0; k < K; k++) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s[k], s[k + 1]);
        kernel_ms[k] += ms;
      }
    }
    float tot = 0.f;
    cudaEventElapsedTime(&tot, ev[0], ev[(n - 1) * (K + 1) + K]);
    *total_ms = tot;
  }
  for (size_t i = 0; i < made; i++) cudaEventDestroy(ev[i]);
  free(ev);
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return read_err(h);
}

int lbm_imb_launches_per_step(lbm_imb_t* h, int* launches) {
  if (!h || !launches) return LBM_IMB_EINVAL;
  if (h->is_batch) {
    *launches = 1;
    return LBM_IMB_OK;
  }
  if (h->is_slab) {  // per slab: clear, raster, collide; then the halo copy and the DEM
    *launches = (h->np > 0 ? 3 : 1) * h->nm + 1 + (h->np > 0 ? 4 * h->v.substeps : 0);
    return LBM_IMB_OK;
  }
  *launches = h->np > 0 ? 3 + (h->v.dem_skin > 0.0 ? 6 : 4) * h->v.substeps : 1;
  return LBM_IMB_OK;
}

int lbm_imb_dem_rebuilds(lbm_imb_t* h, int64_t* builds) {
  if (!h || !builds || h->is_batch) return LBM_IMB_EINVAL;
  long long b = 0;
  if (cudaMemcpyAsync(&b, h->v.vl_builds, 8, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return LBM_IMB_ECUDA;
  *builds = b;
  return LBM_IMB_OK;
}

int lbm_imb_sync(lbm_imb_t* h) {
  if (!h) return LBM_IMB_EINVAL;
  if (h->is_batch) return batch_read_err(h);
  return read_err(h);
}

int lbm_imb_particles(lbm_imb_t* h, double* pos, double* vel, double* omega, double* force,
                      double* torque, int64_t cap) {
  if (!h || cap < h->np) return LBM_IMB_EINVAL;
  const size_t b = 24ull * h->np;
  cudaError_t e = cudaSuccess;
  if (h->np > 0) {
    if (pos) e = e ? e : cudaMemcpyAsync(pos, h->v.pos, b, cudaMemcpyDeviceToHost, h->stream);
    if (vel) e = e ? e : cudaMemcpyAsync(vel, h->v.vel, b, cudaMemcpyDeviceToHost, h->stream);
    if (omega) e = e ? e : cudaMemcpyAsync(omega, h->v.omg, b, cudaMemcpyDeviceToHost, h->stream);
    if (force) e = e ? e : cudaMemcpyAsync(force, h->v.ff, b, cudaMemcpyDeviceToHost, h->stream);
    if (torque) e = e ? e : cudaMemcpyAsync(torque, h->v.tf, b, cudaMemcpyDeviceToHost, h->stream);
  }
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return read_err(h);
}

int lbm_imb_set_particles(lbm_imb_t* h, const double* pos, const double* vel, const double* omega,
                          int64_t n) {
  if (!h || n != h->np) return LBM_IMB_EINVAL;
  const View& gv = h->v;  // ny_glob: the whole lattice's rows (also for a slab)
  const int ext[3] = {gv.nx, gv.ny_glob, gv.nz};
  const int st = check_particle_state(h->dim, ext, gv.wall_y, n, pos, vel, omega);
  if (st) return st;
  const size_t b = 24ull * h->np;
  cudaError_t e = cudaSuccess;
  if (h->np > 0) {
    if (pos) e = e ? e : cudaMemcpyAsync(h->v.pos, pos, b, cudaMemcpyHostToDevice, h->stream);
    if (vel) e = e ? e : cudaMemcpyAsync(h->v.vel, vel, b, cudaMemcpyHostToDevice, h->stream);
    if (omega) e = e ? e : cudaMemcpyAsync(h->v.omg, omega, b, cudaMemcpyHostToDevice, h->stream);
    e = e ? e : cudaStreamSynchronize(h->stream);
  }
  return check_cuda(e);
}

int lbm_imb_fields(lbm_imb_t* h, double* rho, double* u, double* eps, int64_t cap, int on_device) {
  if (h && h->is_slab) return LBM_IMB_EUNSUPPORTED;  // per slab: the member handles
  if (!h || cap < h->N) return LBM_IMB_EINVAL;
  View v = view_of(h, h->cur);
  if (eps) {
    // solid fraction at the current particle positions
    lbm::launch_eps_clear(v, false, h->stream);
    lbm::launch_eps_raster(v, h->smem, h->stream);
  }
  const long long rows = (long long)v.ny * v.nz;
  if (on_device) {
    lbm::launch_fields(v, 0, rows, rho, u, eps, h->stream);
    return check_cuda(cudaGetLastError());
  }
  const int comps = 1 + h->dim + 1;
  const long long chunk = rows_per_chunk(h, comps);
  cudaError_t e = cudaSuccess;
  for (long long r0 = 0; r0 < rows && e == cudaSuccess; r0 += chunk) {
    const long long nr = rows - r0 < chunk ? rows - r0 : chunk;
    const long long cn = nr * v.nx;
    double* srho = h->stage;
    double* su = h->stage + cn;
    double* seps = su + (long long)h->dim * cn;
    lbm::launch_fields(v, r0, nr, rho ? srho : nullptr, u ? su : nullptr, eps ? seps : nullptr, h->stream);
    e = cudaGetLastError();
    const long long off = r0 * v.nx;
    if (rho && e == cudaSuccess)
      e = cudaMemcpyAsync(rho + off, srho, 8 * cn, cudaMemcpyDeviceToHost, h->stream);
    for (int d = 0; u && d < h->dim && e == cudaSuccess; d++)
      e = cudaMemcpyAsync(u + d * h->N + off, su + d * cn, 8 * cn, cudaMemcpyDeviceToHost, h->stream);
    if (eps && e == cudaSuccess)
      e = cudaMemcpyAsync(eps + off, seps, 8 * cn, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return read_err(h);
}

int lbm_imb_get_populations(lbm_imb_t* h, double* f, int64_t cap, int on_device) {
  if (h && h->is_slab) return LBM_IMB_EUNSUPPORTED;  // per slab: the member handles
  if (!h || !f || cap < (int64_t)h->Q * h->N) return LBM_IMB_EINVAL;
  View v = view_of(h, h->cur);
  const long long rows = (long long)v.ny * v.nz;
  if (on_device) {
    lbm::launch_get_populations(v, h->f[h->cur], 0, rows, f, h->stream);
    return check_cuda(cudaGetLastError());
  }
  const long long chunk = rows_per_chunk(h, h->Q);
  cudaError_t e = cudaSuccess;
  for (long long r0 = 0; r0 < rows && e == cudaSuccess; r0 += chunk) {
    const long long nr = rows - r0 < chunk ? rows - r0 : chunk;
    const long long cn = nr * v.nx;
    lbm::launch_get_populations(v, h->f[h->cur], r0, nr, h->stage, h->stream);
    e = cudaGetLastError();
    for (int q = 0; q < h->Q && e == cudaSuccess; q++)
      e = cudaMemcpyAsync(f + q * h->N + r0 * v.nx, h->stage + q * cn, 8 * cn, cudaMemcpyDeviceToHost,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  return check_cuda(e);
}

int lbm_imb_set_populations(lbm_imb_t* h, const double* f, int64_t cap, int on_device) {
  if (h && h->is_slab) return LBM_IMB_EUNSUPPORTED;  // per slab: the member handles
  if (!h || !f || cap < (int64_t)h->Q * h->N) return LBM_IMB_EINVAL;
  View v = view_of(h, h->cur);
  const long long rows = (long long)v.ny * v.nz;
  if (on_device) {
    lbm::launch_set_populations(v, h->f[h->cur], 0, rows, f, h->stream);
    return check_cuda(cudaGetLastError());
  }
  const long long chunk = rows_per_chunk(h, h->Q);
  cudaError_t e = cudaSuccess;
  for (long long r0 = 0; r0 < rows && e == cudaSuccess; r0 += chunk) {
    const long long nr = rows - r0 < chunk ? rows - r0 : chunk;
    const long long cn = nr * v.nx;
    for (int q = 0; q < h->Q && e == cudaSuccess; q++)
      e = cudaMemcpyAsync(h->stage + q * cn, f + q * h->N + r0 * v.nx, 8 * cn, cudaMemcpyHostToDevice,
                          h->stream);
    if (e == cudaSuccess) {
      lbm::launch_set_populations(v, h->f[h->cur], r0, nr, h->stage, h->stream);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  return check_cuda(e);
}

int lbm_imb_totals(lbm_imb_t* h, double* fluid_mass, double* fluid_momentum, double* particle_momentum) {
  if (h && h->is_slab) return LBM_IMB_EUNSUPPORTED;  // per slab: the member handles
  if (!h) return LBM_IMB_EINVAL;
  View v = view_of(h, h->cur);
  lbm::launch_totals(v, h->f[h->cur], h->stream);
  double red[8];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(red, v.red, sizeof(red), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  if (fluid_mass) *fluid_mass = red[0];
  for (int d = 0; d < 3; d++) {
    if (fluid_momentum) fluid_momentum[d] = red[1 + d];
    if (particle_momentum) particle_momentum[d] = red[4 + d];
  }
  if (!isfinite(red[0])) return LBM_IMB_ENONFINITE;
  return read_err(h);
}

int lbm_imb_drag_samples(lbm_imb_t* h, const double* u_dev, const double* eps_dev, double shell, float* feats,
                         float* target, int64_t cap) {
  if (!h || h->is_batch || h->is_slab || !u_dev || !eps_dev || !feats || !target || cap < h->np || !(shell > 0.0))
    return LBM_IMB_EINVAL;
  View v = view_of(h, h->cur);
  lbm::launch_drag_samples(v, u_dev, eps_dev, shell, feats, target, h->stream);
  return check_cuda(cudaGetLastError());
}

int lbm_imb_set_collide_variant(lbm_imb_t* h, int variant) {
  if (h && h->is_slab) return LBM_IMB_EUNSUPPORTED;  // per slab: the member handles
  if (!h || h->is_member || variant < 0 || variant > 9) return LBM_IMB_EINVAL;
  if (h->is_batch) return LBM_IMB_EUNSUPPORTED;
  if (h->graphs_ok) {
    cudaGraphExecDestroy(h->graph[0]);
    cudaGraphExecDestroy(h->graph[1]);
  }
  h->graphs_ok = false;
  h->graphs_tried = false;
  h->v.collide_variant = variant;
  return LBM_IMB_OK;
}

int lbm_imb_set_health_check(lbm_imb_t* h, int64_t every) {
  if (!h || h->is_member || every < 0) return LBM_IMB_EINVAL;
  h->health_every = every;
  return LBM_IMB_OK;
}

int lbm_imb_check_health(lbm_imb_t* h) {
  if (!h || h->is_member) return LBM_IMB_EINVAL;
  enqueue_health(h);
  if (cudaGetLastError() != cudaSuccess) return LBM_IMB_ECUDA;
  return h->is_batch ? batch_read_err(h) : read_err(h);
}

// ---- checkpoints ----
// File: a fixed header, then the stored populations of the current lattice
// (raw storage bytes, Q planes of pitch * ny * nz elements), then the
// particle arrays pos, vel, omega, force, torque ([n][3] FP64 each).
namespace {
struct CkptHeader {
  char magic[8];        // "LBMIMBCK"
  uint32_t version;     // 1
  uint32_t header_bytes;
  uint64_t cfg_hash;
  int32_t dim, nx, ny, nz, Q, storage, pitch, esz;
  int64_t np, steps;
  uint64_t pop_bytes, particle_bytes;
};
constexpr char kCkptMagic[8] = {'L', 'B', 'M', 'I', 'M', 'B', 'C', 'K'};

void ckpt_header(const lbm_imb* h, CkptHeader* H) {
  memset(H, 0, sizeof(*H));
  memcpy(H->magic, kCkptMagic, 8);
  H->version = 1;
  H->header_bytes = sizeof(CkptHeader);
  H->cfg_hash = h->cfg_hash;
  H->dim = h->dim;
  H->nx = h->v.nx;
  H->ny = h->v.ny;
  H->nz = h->v.nz;
  H->Q = h->Q;
  H->storage = h->v.storage;
  H->pitch = h->v.pitch;
  H->esz = lbm::pop_bytes(h->v.storage);
  H->np = h->np;
  H->steps = h->steps;
  H->pop_bytes = (uint64_t)h->Q * (uint64_t)h->v.plane * (uint64_t)H->esz;
  H->particle_bytes = 5ull * 24ull * (uint64_t)h->np;
}

// device range <-> file through the staging area, in chunks
int ckpt_copy(lbm_imb* h, FILE* fp, unsigned char* dev, uint64_t bytes, bool to_file) {
  unsigned char* buf = static_cast<unsigned char*>(malloc(h->stage_bytes));
  if (!buf) return LBM_IMB_ENOMEM;
  int st = LBM_IMB_OK;
  for (uint64_t o = 0; o < bytes && !st; o += h->stage_bytes) {
    const size_t n = (size_t)(bytes - o < h->stage_bytes ? bytes - o : h->stage_bytes);
    if (to_file) {
      if (cudaMemcpyAsync(buf, dev + o, n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
          cudaStreamSynchronize(h->stream) != cudaSuccess)
        st = LBM_IMB_ECUDA;
      else if (fwrite(buf, 1, n, fp) != n)
        st = LBM_IMB_EINVAL;
    } else {
      if (fread(buf, 1, n, fp) != n)
        st = LBM_IMB_EINVAL;
      else if (cudaMemcpyAsync(dev + o, buf, n, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
               cudaStreamSynchronize(h->stream) != cudaSuccess)
        st = LBM_IMB_ECUDA;
    }
  }
  free(buf);
  return st;
}

double* particle_array(lbm_imb* h, int k) {
  double* a[5] = {h->v.pos, h->v.vel, h->v.omg, h->v.ff, h->v.tf};
  return a[k];
}
}  // namespace

int lbm_imb_save(lbm_imb_t* h, const char* path) {
  if (!h || !path || h->is_batch || h->is_slab || h->is_member) return h && path ? LBM_IMB_EUNSUPPORTED
                                                                                     : LBM_IMB_EINVAL;
  int st = read_err(h);  // a failed run is not saved
  if (st) return st;
  CkptHeader H;
  ckpt_header(h, &H);
  FILE* fp = fopen(path, "wb");
  if (!fp) return LBM_IMB_EINVAL;
  if (fwrite(&H, sizeof(H), 1, fp) != 1) st = LBM_IMB_EINVAL;
  if (!st) st = ckpt_copy(h, fp, static_cast<unsigned char*>(h->f[h->cur]), H.pop_bytes, true);
  for (int k = 0; k < 5 && !st && h->np > 0; k++)
    st = ckpt_copy(h, fp, reinterpret_cast<unsigned char*>(particle_array(h, k)), 24ull * h->np, true);
  if (fclose(fp) != 0 && !st) st = LBM_IMB_EINVAL;
  return st;
}

int lbm_imb_load(lbm_imb_t* h, const char* path) {
  if (!h || !path || h->is_batch || h->is_slab || h->is_member) return h && path ? LBM_IMB_EUNSUPPORTED
                                                                                     : LBM_IMB_EINVAL;
  int st = read_err(h);
  if (st) return st;
  CkptHeader want, got;
  ckpt_header(h, &want);
  FILE* fp = fopen(path, "rb");
  if (!fp) return LBM_IMB_EINVAL;
  if (fread(&got, sizeof(got), 1, fp) != 1 || memcmp(got.magic, kCkptMagic, 8) != 0 || got.version != 1 ||
      got.header_bytes != sizeof(CkptHeader) || got.cfg_hash != want.cfg_hash || got.dim != want.dim ||
      got.nx != want.nx || got.ny != want.ny || got.nz != want.nz || got.Q != want.Q ||
      got.storage != want.storage || got.pitch != want.pitch || got.esz != want.esz || got.np != want.np ||
      got.pop_bytes != want.pop_bytes || got.particle_bytes != want.particle_bytes || got.steps < 0) {
    fclose(fp);
    return LBM_IMB_EINVAL;
  }
  st = ckpt_copy(h, fp, static_cast<unsigned char*>(h->f[h->cur]), got.pop_bytes, false);
  for (int k = 0; k < 5 && !st && h->np > 0; k++)
    st = ckpt_copy(h, fp, reinterpret_cast<unsigned char*>(particle_array(h, k)), 24ull * h->np, false);
  fclose(fp);
  if (st) return st;
  // Verlet lists (dem_skin > 0) are rebuilt from the loaded positions at the
  // next step: the same pairs, so the same contact forces
  if (h->v.dem_skin > 0.0) {
    const int one = 1;
    if (cudaMemcpyAsync(h->v.vl_flag, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return LBM_IMB_ECUDA;
  }
  h->steps = got.steps;
  return LBM_IMB_OK;
}

int lbm_imb_steps_done(lbm_imb_t* h, int64_t* steps) {
  if (!h || !steps) return LBM_IMB_EINVAL;
  *steps = h->steps;
  return LBM_IMB_OK;
}

int lbm_imb_destroy(lbm_imb_t* h) {
  if (!h || h->is_member) return LBM_IMB_EINVAL;
  if (h->is_batch) {
    batch_drop_graphs(h);
    for (int i = 0; i < h->nm; i++) lbm_imb_destroy_member_graphs(h->members + i);
    delete[] h->members;
    delete h;
    return LBM_IMB_OK;
  }
  if (h->is_slab) {
    if (h->graphs_ok) {
      cudaGraphExecDestroy(h->graph[0]);
      cudaGraphExecDestroy(h->graph[1]);
    }
    delete[] h->members;
    delete h;
    return LBM_IMB_OK;
  }
  if (h->graphs_ok) {
    cudaGraphExecDestroy(h->graph[0]);
    cudaGraphExecDestroy(h->graph[1]);
  }
  delete h;
  return LBM_IMB_OK;
}

const char* lbm_imb_strerror(int s) {
  switch (s) {
    case LBM_IMB_OK: return "ok";
    case LBM_IMB_EINVAL: return "invalid argument or configuration";
    case LBM_IMB_ENOMEM: return "device block smaller than lbm_imb_required_bytes";
    case LBM_IMB_ECUDA: return "CUDA runtime error";
    case LBM_IMB_ETIMEOUT: return "a bounded device wait timed out";
    case LBM_IMB_ENONFINITE: return "non-finite value found";
    case LBM_IMB_EUNSUPPORTED: return "configuration outside the implemented limits";
    case LBM_IMB_EOWNERS: return "a lattice cell was covered by more particles than supported";
    case LBM_IMB_EBIN: return "a DEM cell-list bin or contact list overflowed";
    default: return "unknown status";
  }
}

// ---- standalone DEM contact forces ----
namespace {
struct DemWs {
  size_t off_err, off_binof, off_count, off_slot, total;
  int nb[3];
  double bsz[3];
};
int dem_ws_layout(int32_t dim, const int32_t* extent, int32_t wall_y, int64_t n, double rmax, DemWs* w) {
  if ((dim != 2 && dim != 3) || !extent || n < 0 || n > (1ll << 30) || !(rmax > 0.0)) return LBM_IMB_EINVAL;
  if (wall_y != 0 && wall_y != 1) return LBM_IMB_EINVAL;
  int ext[3] = {extent[0], extent[1], dim == 3 ? extent[2] : 1};
  for (int d = 0; d < 3; d++)
    if (ext[d] < 1) return LBM_IMB_EINVAL;
  int st = lbm::dem_bin_geometry(dim, ext, wall_y, rmax, w->nb, w->bsz);
  if (st) return st;
  const size_t nbins = (size_t)w->nb[0] * w->nb[1] * w->nb[2];
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  w->off_err = take(16);
  w->off_binof = take((size_t)(n > 0 ? n : 1) * 4);
  w->off_count = take(nbins * 4);
  w->off_slot = take(nbins * lbm::kBinCap * 4);
  w->total = o;
  return LBM_IMB_OK;
}
}  // namespace

size_t lbm_imb_dem_workspace_bytes(int32_t dim, const int32_t* extent, int32_t wall_y, int64_t n, double rmax) {
  DemWs w;
  if (dem_ws_layout(dim, extent, wall_y, n, rmax, &w) != LBM_IMB_OK) return 0;
  return w.total;
}

int lbm_imb_dem_forces(int32_t dim, const int32_t* extent, int32_t wall_y, int64_t n, double rmax,
                       const double* pos, const double* vel, const double* radius, const double* mass,
                       double k_n, double restitution, double* fc, void* workspace, size_t workspace_bytes,
                       void* stream) {
  if (n > 0 && (!pos || !vel || !radius || !mass || !fc)) return LBM_IMB_EINVAL;
  if (!workspace || ((uintptr_t)workspace) % kAlign) return LBM_IMB_EINVAL;
  if (!(k_n >= 0.0) || !(restitution > 0.0 && restitution <= 1.0)) return LBM_IMB_EINVAL;
  if (n == 0) return LBM_IMB_OK;
  DemWs w;
  int st = dem_ws_layout(dim, extent, wall_y, n, rmax, &w);
  if (st) return st;
  if (workspace_bytes < w.total) return LBM_IMB_ENOMEM;
  unsigned char* base = static_cast<unsigned char*>(workspace);
  View v;
  memset(&v, 0, sizeof(v));
  v.dim = dim;
  v.nx = extent[0];
  v.ny = extent[1];
  v.nz = dim == 3 ? extent[2] : 1;
  v.wall_y = wall_y;
  v.np = (int)n;
  v.pos = const_cast<double*>(pos);
  v.vel = const_cast<double*>(vel);
  v.rad = const_cast<double*>(radius);
  v.mass = const_cast<double*>(mass);
  v.fc = fc;
  v.err = reinterpret_cast<int*>(base + w.off_err);
  v.bin_of = reinterpret_cast<int*>(base + w.off_binof);
  v.bin_count = reinterpret_cast<int*>(base + w.off_count);
  v.bin_slot = reinterpret_cast<int*>(base + w.off_slot);
  for (int d = 0; d < 3; d++) {
    v.nb[d] = w.nb[d];
    v.bsz[d] = w.bsz[d];
  }
  v.kn = k_n;
  const double le = log(restitution);
  v.ln_e = le;
  v.dem_den = M_PI * M_PI + le * le;
  v.substeps = 1;
  v.rmax_bins = rmax;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(v.err, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    lbm::launch_dem_contacts(v, s);
    e = cudaGetLastError();
  }
  int bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, v.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LBM_IMB_ECUDA;
  return map_err(bits);
}

const char* lbm_imb_version(void) { return "lbm_imb 0.1 (sm_103a)"; }

}  // extern "C"
