// Internal declarations shared by the CUDA translation units of liblbm_imb.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbm_imb.h"

namespace lbm {

constexpr int kMaxOwners = LBM_IMB_MAX_OWNERS;
constexpr int kBinCap = 16;  // particles per DEM cell-list bin
constexpr int kVerletCap = 48;  // partners per Verlet list

// device error word bits
enum : int { ERR_OWNERS = 1, ERR_BIN = 2, ERR_NONFINITE = 4, ERR_TIMEOUT = 8 };

// status of a device error word (the most severe condition first)
inline int status_of_err_bits(int bits) {
  if (bits & ERR_TIMEOUT) return LBM_IMB_ETIMEOUT;
  if (bits & ERR_OWNERS) return LBM_IMB_EOWNERS;
  if (bits & ERR_BIN) return LBM_IMB_EBIN;
  if (bits & ERR_NONFINITE) return LBM_IMB_ENONFINITE;
  return LBM_IMB_OK;
}

// largest |coordinate| of a particle centre the kernels index with (lattice
// units); beyond it (or NaN/Inf) the particle is reported as ERR_NONFINITE
// and skipped, which keeps every box origin and extent inside int range
constexpr double kPosLimit = 1073741824.0;  // 2^30

// ---------------------------------------------------------------------------
// Lattice descriptors (interface direction order: rest, then opposite pairs).
// All loops over directions are unrolled, so every lookup folds to a literal.
// ---------------------------------------------------------------------------
struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int DIM = 2;
  __host__ __device__ static constexpr int c(int q, int d) {
    constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0},   {-1, 0, 0},
                             {0, 1, 0}, {0, -1, 0},  {1, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    return t[q][d];
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int DIM = 3;
  __host__ __device__ static constexpr int c(int q, int d) {
    constexpr int t[19][3] = {
        {0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
        {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
        {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    return t[q][d];
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 1.0 / 3.0 : (q < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

// opposite direction: pairs (1,2), (3,4), ...
__host__ __device__ constexpr int opp(int q) {
  return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1);
}

// ---------------------------------------------------------------------------
// Device view of one simulation (passed by value to kernels).
// ---------------------------------------------------------------------------
struct View {
  // lattice geometry
  int dim, Q, nx, ny, nz, pitch, wall_y, storage;
  // y slab of a decomposed lattice: local rows y0 .. y0 + ny_c - 1 are
  // computed (the rows around them are halos the exchange fills); local row
  // y is row y + ygo of the whole lattice, ny_glob rows tall; a wall lies
  // below the first / above the last computed row when wall_lo / wall_hi.
  // A whole lattice: y0 = 0, ny_c = ny, ygo = 0, ny_glob = ny,
  // wall_lo = wall_hi = wall_y.
  int y0, ny_c, ygo, ny_glob, wall_lo, wall_hi;
  long long plane;  // elements per population plane = pitch * ny * nz
  // populations: src is read (pull), dst written; per-direction plane
  // bases (fsrc + q * plane elements), filled by the host with fsrc/fdst
  void* fsrc;
  void* fdst;
  const void* src_q[19];
  void* dst_q[19];
  // solid-fraction slots; eps element type follows the storage (double for
  // F64, float otherwise)
  int* own[kMaxOwners];
  void* eps[kMaxOwners];
  // particles (FP64 SoA-of-vec3)
  int np;
  double *pos, *vel, *omg, *rad, *mass, *inertia;
  double *ff, *tf, *fc;  // hydrodynamic force/torque (Eq. 3), contact force
  int* lo;               // [np*6] origin and extent of the last rasterised box
  float* kin;            // [np*16] FP32 kinematics: frac pos, int pos, v, omega
  int* bin_of;           // [np] DEM bin of each particle
  // DEM bins
  int nb[3];
  double bsz[3];
  int* bin_count;  // [nbins]
  int* bin_slot;   // [nbins * kBinCap]
  double rmax_bins;  // largest radius the bins were sized for
  // Verlet neighbour lists (dem_skin > 0): [np][kVerletCap] partner ids in
  // ascending order, their counts, the positions at the last build, and
  // flag[0] = rebuild needed, *builds = number of builds
  double dem_skin;
  int* vl_nbr;
  int* vl_count;
  double* vl_ref;
  int* vl_flag;
  long long* vl_builds;
  // covered-node list of the split collision (pair storage, form
  // kCollideSplit): the rasteriser appends every node whose first owner slot
  // it claims; null otherwise
  int* cov_list;
  int* cov_count;
  // compact buffer of the split form kCollideSplit + 3 (pair storage): the
  // plain kernel appends each covered node's pulled populations and moments
  // (pairs as float2, SoA [Q + 5][cbuf_cap]), first covered fraction
  // (double [cbuf_cap]), node offset and first two owner slots (int
  // [3][cbuf_cap]), counted in cov_count; null otherwise
  float2* cbuf;
  long long cbuf_cap;
  // physics
  double tau, omega, gf[3], gs[3], rho0, kn, ln_e, dem_den;
  double fq[19];  // 3 w_q (c_q . g_f): body force per unit density, Eq. (1) F_i
  double cg3[19];  // 3 c_q . g_f
  double omc;     // 1 - omega
  // FP32 copies for the reduced-precision kernels (a double -> float
  // conversion runs on the FP64 pipe, so none happens per node)
  float tau_f, omega_f, rho0_f, omc_f;
  float fq_f[19], cg3_f[19];
  // the same as FP32 pairs (high, low) for the double-FP32 collision
  float tau_df[2], omega_df[2], rho0_df[2], omc_df[2];
  float fq_df[19][2], cg3_df[19][2];
  int substeps;
  int collide_variant;  // kernel form of the collision
  // covered fractions: 0 exact closed forms, 1 the Eq. 6 table (one radius)
  int eps_method;
  const float* eps_tab;  // table of exact fractions (see dev_eps.cuh)
  float tab_lo_r, tab_h_r, tab_h_s, tab_h_t;
  // device error word
  int* err;
  // scratch for reductions (totals)
  double* red;
};

static_assert(sizeof(View) % sizeof(int) == 0, "View is copied as ints");

// collide forms of the pair storage that update plain and covered nodes in
// two launches (the covered ones from the rasteriser's list): covered nodes
// in FP64 (kCollideSplit) or in pair arithmetic (kCollideSplit + 1, and + 2
// with the plain part two nodes per thread)
constexpr int kCollideSplit = 6;
__host__ __device__ inline bool split_form(int variant) {
  return variant >= kCollideSplit && variant <= kCollideSplit + 2;
}

// bytes of one stored population; whether the covered fractions (and the
// rasteriser) are FP64
__host__ __device__ inline int pop_bytes(int storage) {
  return (storage == LBM_IMB_STORE_F64 || storage == LBM_IMB_STORE_DFDEV) ? 8
         : storage == LBM_IMB_STORE_F32DEV                                 ? 4
                                                                           : 2;
}
__host__ __device__ inline bool fp64_eps(int storage) { return storage == LBM_IMB_STORE_F64 || storage == LBM_IMB_STORE_DFDEV; }

// ---------------------------------------------------------------------------
// Launchers (one per kernel family; each in its own translation unit).
// ---------------------------------------------------------------------------
void launch_init_equilibrium(const View& v, void* f, cudaStream_t s);
void launch_eps_clear(const View& v, bool zero_forces, cudaStream_t s);
void launch_eps_raster(const View& v, int smem_bytes, cudaStream_t s);
int eps_raster_smem_bytes(int dim, int storage, double rmax);
int eps_table_raster_smem_bytes(int dim, int storage, double rmax);
long long eps_table_entries(int dim);
void eps_table_geometry(int dim, double R, float* lo_r, float* h_r, float* h_s, float* h_t);
cudaError_t launch_eps_table_build(int dim, double R, float* tab, cudaStream_t s);
int eps_raster_set_attrs(int bytes);
void launch_collide(const View& v, cudaStream_t s);
// halo rows of y slabs: for every boundary, the last computed row of the
// lower slab and the first of the upper one are copied (all directions, all
// z) into the other slab's halo row of the populations `parity`
struct SlabHalo {
  unsigned char* f[2][16];  // per slab: the two population lattices
  int ny[16];               // per slab: local rows (computed + 2 halos)
  int ns;                   // slabs
  int periodic;             // exchange across the ends too (no walls)
  long long plane_bytes[16];
  int row_bytes, nz;
  // the directions a halo row feeds: qdir[0] those with c_y = +1 (pulled
  // from the row below the first computed row), qdir[1] those with c_y = -1
  int nq, qdir[2][8];
};
cudaError_t launch_halo_exchange(const SlabHalo& h, int parity, cudaStream_t s);
void launch_dem(const View& v, cudaStream_t s);
void launch_dem_contacts(const View& v, cudaStream_t s);
int dem_bin_geometry(int dim, const int* ext, int wall_y, double rmax, int nb[3], double bsz[3]);
void launch_fields(const View& v, long long row0, long long nrows, double* rho, double* u, double* eps,
                   cudaStream_t s);
void launch_get_populations(const View& v, const void* f, long long row0, long long nrows, double* out,
                            cudaStream_t s);
void launch_set_populations(const View& v, void* f, long long row0, long long nrows, const double* in,
                            cudaStream_t s);
void launch_totals(const View& v, const void* f, cudaStream_t s);
// health check: non-finite stored rest populations or particle state set
// ERR_NONFINITE in the error word
void launch_health(const View& v, const void* f, cudaStream_t s);
void launch_drag_samples(const View& v, const double* u, const double* eps, double shell, float* feats,
                         float* target, cudaStream_t s);

}  // namespace lbm
