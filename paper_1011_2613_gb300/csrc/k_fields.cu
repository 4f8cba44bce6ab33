// K4: initial equilibrium, macroscopic fields, population import/export and
// global sums.  The fields are the moments of the populations the next
// collision sees (the stored post-collision state pulled one step, as in K2),
// with the fluid velocity u = sum_i f_i c_i / rho + g_f / 2.
#include "dev_df.cuh"
#include "lbm_internal.cuh"

namespace lbm {

// stored value <-> FP64 population
__device__ __forceinline__ double stored_to_f(const void* f, int storage, long long i, double w,
                                              double rho0) {
  if (storage == LBM_IMB_STORE_F64) return static_cast<const double*>(f)[i];
  if (storage == LBM_IMB_STORE_DFDEV) {
    const float2 p = static_cast<const float2*>(f)[i];
    return w * rho0 + ((double)p.x + (double)p.y);
  }
  if (storage == LBM_IMB_STORE_F32DEV) return w * rho0 + (double)static_cast<const float*>(f)[i];
  return w * rho0 + w * (double)__half2float(static_cast<const __half*>(f)[i]);
}
__device__ __forceinline__ void f_to_stored(void* f, int storage, long long i, double w, double rho0,
                                            double val) {
  if (storage == LBM_IMB_STORE_F64) static_cast<double*>(f)[i] = val;
  else if (storage == LBM_IMB_STORE_DFDEV) {
    const double g = val - w * rho0;
    const float h = (float)g;
    static_cast<float2*>(f)[i] = make_float2(h, (float)(g - (double)h));
  }
  else if (storage == LBM_IMB_STORE_F32DEV) static_cast<float*>(f)[i] = (float)(val - w * rho0);
  else static_cast<__half*>(f)[i] = __float2half_rn((float)((val - w * rho0) / w));
}

template <class LAT>
__global__ void init_eq_kernel(View v, void* f) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= v.plane) return;
#pragma unroll
  for (int q = 0; q < LAT::Q; q++)
    f_to_stored(f, v.storage, q * v.plane + i, LAT::w(q), v.rho0, LAT::w(q) * v.rho0);
}

// Rows are (y, z) pairs flattened as r = z * ny + y; a launch covers rows
// [row0, row0 + nrows) and writes dense outputs relative to row0 with
// component stride nrows * nx (so large fields can be staged in chunks).
template <class LAT>
__global__ void fields_kernel(View v, long long row0, long long nrows, double* rho_out,
                              double* u_out, double* eps_out) {
  const long long r = row0 + blockIdx.x;
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= v.nx) return;
  const int nx = v.nx, ny = v.ny, nz = v.nz;
  const int y = (int)(r % ny), z = (int)(r / ny);
  const long long n = r * v.pitch + x;
  const long long dense = (r - row0) * nx + x;
  const long long N = nrows * nx;
  double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < LAT::Q; q++) {
    const int cx = LAT::c(q, 0), cy = LAT::c(q, 1), cz = LAT::c(q, 2);
    const int sx = (x - cx + nx) % nx;
    const int sz = (z - cz + nz) % nz;
    int sy = y - cy;
    double val;
    if (v.wall_y && (sy < 0 || sy >= ny)) {
      val = stored_to_f(v.fsrc, v.storage, opp(q) * v.plane + n, LAT::w(opp(q)), v.rho0);
    } else {
      sy = (sy + ny) % ny;
      val = stored_to_f(v.fsrc, v.storage, q * v.plane + ((long long)sz * ny + sy) * v.pitch + sx,
                        LAT::w(q), v.rho0);
    }
    rho += val;
    j[0] += val * cx;
    j[1] += val * cy;
    j[2] += val * cz;
  }
  if (rho_out) rho_out[dense] = rho;
  if (u_out)
    for (int d = 0; d < LAT::DIM; d++) u_out[d * N + dense] = j[d] / rho + 0.5 * v.gf[d];
  if (eps_out) {
    double es = 0.0;
    for (int s = 0; s < kMaxOwners; s++) {
      if (v.own[s][n] < 0) break;
      es += fp64_eps(v.storage) ? static_cast<const double*>(v.eps[s])[n]
                                           : (double)static_cast<const float*>(v.eps[s])[n];
    }
    eps_out[dense] = es < 1.0 ? es : 1.0;
  }
}

template <class LAT>
__global__ void get_pop_kernel(View v, const void* f, long long row0, long long nrows, double* out) {
  const long long r = row0 + blockIdx.x;
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= v.nx) return;
  const long long n = r * v.pitch + x;
  const long long dense = (r - row0) * v.nx + x;
  const long long N = nrows * v.nx;
#pragma unroll
  for (int q = 0; q < LAT::Q; q++)
    out[q * N + dense] = stored_to_f(f, v.storage, q * v.plane + n, LAT::w(q), v.rho0);
}

template <class LAT>
__global__ void set_pop_kernel(View v, void* f, long long row0, long long nrows, const double* in) {
  const long long r = row0 + blockIdx.x;
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= v.nx) return;
  const long long n = r * v.pitch + x;
  const long long dense = (r - row0) * v.nx + x;
  const long long N = nrows * v.nx;
#pragma unroll
  for (int q = 0; q < LAT::Q; q++)
    f_to_stored(f, v.storage, q * v.plane + n, LAT::w(q), v.rho0, in[q * N + dense]);
}

// red[0] = mass, red[1..3] = fluid momentum, red[4..6] = particle momentum
template <class LAT>
__global__ void totals_kernel(View v, const void* f) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  double m = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
  if (x < v.nx) {
    const long long n = ((long long)z * v.ny + y) * v.pitch + x;
#pragma unroll
    for (int q = 0; q < LAT::Q; q++) {
      const double val = stored_to_f(f, v.storage, q * v.plane + n, LAT::w(q), v.rho0);
      m += val;
      j0 += val * LAT::c(q, 0);
      j1 += val * LAT::c(q, 1);
      j2 += val * LAT::c(q, 2);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_down_sync(0xffffffffu, m, o);
    j0 += __shfl_down_sync(0xffffffffu, j0, o);
    j1 += __shfl_down_sync(0xffffffffu, j1, o);
    j2 += __shfl_down_sync(0xffffffffu, j2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(v.red, m);
    atomicAdd(v.red + 1, j0);
    atomicAdd(v.red + 2, j1);
    atomicAdd(v.red + 3, j2);
  }
}

__global__ void particle_momentum_kernel(View v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.np) return;
  for (int d = 0; d < 3; d++) atomicAdd(v.red + 4 + d, v.mass[i] * v.vel[3 * i + d]);
}

__global__ void zero_red_kernel(double* red) {
  if (threadIdx.x < 8) red[threadIdx.x] = 0.0;
}

// Health check.  A NaN or Inf in any population of a node reaches the
// node's density and velocity, and through them every population the
// collision writes there, the rest direction included; a population that
// streams it elsewhere does the same at the next node one step later.  So
// the stored rest-direction plane (1/Q of the lattice) shows every
// non-finite population within one step of its appearance.  The particle
// state is scanned beside it.  Any hit sets ERR_NONFINITE.
__device__ __forceinline__ bool stored_finite(const void* f, int storage, long long i) {
  if (storage == LBM_IMB_STORE_F64) return isfinite(static_cast<const double*>(f)[i]);
  if (storage == LBM_IMB_STORE_DFDEV) {
    const float2 p = static_cast<const float2*>(f)[i];
    return isfinite(p.x) && isfinite(p.y);
  }
  if (storage == LBM_IMB_STORE_F32DEV) return isfinite(static_cast<const float*>(f)[i]);
  return isfinite(__half2float(static_cast<const __half*>(f)[i]));
}

__global__ void health_kernel(View v, const void* f) {
  bool bad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v.plane; i += stride)
    bad |= !stored_finite(f, v.storage, i);  // direction 0: the first plane
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3LL * v.np; i += stride)
    bad |= !(fabs(v.pos[i]) <= kPosLimit) || !isfinite(v.vel[i]) || !isfinite(v.omg[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(v.err, ERR_NONFINITE);
}

void launch_health(const View& v, const void* f, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long work = v.plane > 3LL * v.np ? v.plane : 3LL * v.np;
  long long blocks = (work + 255) / 256;
  const long long cap = 4LL * (sms > 0 ? sms : 1);
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  health_kernel<<<(unsigned)blocks, 256, 0, s>>>(v, f);
}

void launch_init_equilibrium(const View& v, void* f, cudaStream_t s) {
  const int T = 256;
  const long long blocks = (v.plane + T - 1) / T;
  if (v.dim == 2) init_eq_kernel<D2Q9><<<blocks, T, 0, s>>>(v, f);
  else init_eq_kernel<D3Q19><<<blocks, T, 0, s>>>(v, f);
}

static dim3 row_grid(const View& v) { return dim3((v.nx + 127) / 128, v.ny, v.nz); }
static dim3 chunk_grid(const View& v, long long nrows) { return dim3((unsigned)nrows, (v.nx + 127) / 128, 1); }

void launch_fields(const View& v, long long row0, long long nrows, double* rho, double* u, double* eps,
                   cudaStream_t s) {
  if (v.dim == 2) fields_kernel<D2Q9><<<chunk_grid(v, nrows), 128, 0, s>>>(v, row0, nrows, rho, u, eps);
  else fields_kernel<D3Q19><<<chunk_grid(v, nrows), 128, 0, s>>>(v, row0, nrows, rho, u, eps);
}

void launch_get_populations(const View& v, const void* f, long long row0, long long nrows, double* out,
                            cudaStream_t s) {
  if (v.dim == 2) get_pop_kernel<D2Q9><<<chunk_grid(v, nrows), 128, 0, s>>>(v, f, row0, nrows, out);
  else get_pop_kernel<D3Q19><<<chunk_grid(v, nrows), 128, 0, s>>>(v, f, row0, nrows, out);
}

void launch_set_populations(const View& v, void* f, long long row0, long long nrows, const double* in,
                            cudaStream_t s) {
  if (v.dim == 2) set_pop_kernel<D2Q9><<<chunk_grid(v, nrows), 128, 0, s>>>(v, f, row0, nrows, in);
  else set_pop_kernel<D3Q19><<<chunk_grid(v, nrows), 128, 0, s>>>(v, f, row0, nrows, in);
}

void launch_totals(const View& v, const void* f, cudaStream_t s) {
  zero_red_kernel<<<1, 32, 0, s>>>(v.red);
  if (v.dim == 2) totals_kernel<D2Q9><<<row_grid(v), 128, 0, s>>>(v, f);
  else totals_kernel<D3Q19><<<row_grid(v), 128, 0, s>>>(v, f);
  if (v.np > 0) particle_momentum_kernel<<<(v.np + 127) / 128, 128, 0, s>>>(v);
}

}  // namespace lbm

namespace lbm {

// Halo rows of y slabs (lbm_imb_slabs_init).  Work item = one 16-byte piece
// of one row of one direction plane at one z, for one side of one slab
// boundary: side 0 copies the lower slab's last computed row into the upper
// slab's lower halo, side 1 the upper slab's first computed row into the
// lower slab's upper halo.  Only the directions the pull reads from a halo
// row move: c_y = +1 on side 0, c_y = -1 on side 1 (5 of 19 in D3Q19, 3 of
// 9 in D2Q9).  Rows are whole multiples of 64 bytes (pitch is a multiple of
// 32 elements) and planes start on 256-byte boundaries.
__global__ void halo_exchange_kernel(SlabHalo h, int parity) {
  const int pieces = h.row_bytes / 16;
  const int nbound = h.periodic ? h.ns : h.ns - 1;
  const long long per_side = (long long)h.nq * h.nz * pieces;
  const long long total = 2LL * nbound * per_side;
  for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < total;
       w += (long long)gridDim.x * blockDim.x) {
    const long long bs = w / per_side;
    long long r = w - bs * per_side;
    const int b = (int)(bs >> 1), side = (int)(bs & 1);
    const int iq = (int)(r / ((long long)h.nz * pieces));
    r -= (long long)iq * h.nz * pieces;
    const int z = (int)(r / pieces), c = (int)(r - (long long)z * pieces);
    const int q = h.qdir[side][iq];
    const int lo = b, hi = b + 1 == h.ns ? 0 : b + 1;
    const int from = side == 0 ? lo : hi, to = side == 0 ? hi : lo;
    const int yf = side == 0 ? h.ny[lo] - 2 : 1;   // computed row
    const int yt = side == 0 ? 0 : h.ny[lo] - 1;   // halo row
    const unsigned char* src = h.f[parity][from] + q * h.plane_bytes[from] +
                               ((long long)z * h.ny[from] + yf) * h.row_bytes + 16LL * c;
    unsigned char* dst = h.f[parity][to] + q * h.plane_bytes[to] +
                         ((long long)z * h.ny[to] + yt) * h.row_bytes + 16LL * c;
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
  }
}

cudaError_t launch_halo_exchange(const SlabHalo& h, int parity, cudaStream_t s) {
  const int nbound = h.periodic ? h.ns : h.ns - 1;
  const long long total = 2LL * nbound * h.nq * h.nz * (h.row_bytes / 16);
  if (total <= 0) return cudaSuccess;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  halo_exchange_kernel<<<(unsigned)blocks, 256, 0, s>>>(h, parity);
  return cudaGetLastError();
}

}  // namespace lbm

namespace lbm {

__global__ void df_probe_kernel(const float* h, const float* l, const double* d, double* to_double,
                                double* roundtrip, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  to_double[i] = df_to_bits(DF(h[i], l[i]));
  roundtrip[i] = df_to_bits(df_from_bits(d[i]));
}

}  // namespace lbm

extern "C" int lbm_imb_probe_df(const float* h, const float* l, const double* d, double* to_double,
                                double* roundtrip, int64_t n, void* stream) {
  if (!h || !l || !d || !to_double || !roundtrip || n < 0) return LBM_IMB_EINVAL;
  if (n == 0) return LBM_IMB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  lbm::df_probe_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h, l, d, to_double, roundtrip, (long long)n);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return LBM_IMB_ECUDA;
  return LBM_IMB_OK;
}

namespace lbm {

// FP64 pipe rate: every thread runs 16 independent chains of one FP64
// instruction (KIND 0 fused multiply-add, 1 add, 2 multiply; one FP64-pipe
// operation each), 16 per chain and loop trip; the chains' sums are stored
// so that nothing is optimised away.  The constant operands m and c are
// kernel parameters, read from the constant bank: the only register operand
// is the chain itself, so register-file bandwidth does not cap the rate
// (with m and c in registers a DFMA stream reaches only 0.84 of the pipe)
constexpr int kFp64Chains = 16;
constexpr int kFp64Reps = 16;
template <int KIND>
__global__ void __launch_bounds__(256) fp64_rate_kernel(double* sink, long long trips, double m, double c) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double a[kFp64Chains];
#pragma unroll
  for (int k = 0; k < kFp64Chains; k++) a[k] = 1.0 + 1e-9 * (double)(i + k);
  for (long long t = 0; t < trips; t++) {
#pragma unroll
    for (int r = 0; r < kFp64Reps; r++)
#pragma unroll
      for (int k = 0; k < kFp64Chains; k++) {
        if constexpr (KIND == 0) a[k] = fma(a[k], m, c);
        else if constexpr (KIND == 1) a[k] = __dadd_rn(a[k], c);
        else a[k] = __dmul_rn(a[k], m);
      }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kFp64Chains; k++) s += a[k];
  sink[i] = s;
}

}  // namespace lbm

extern "C" int lbm_imb_probe_fp64_rate(double* dev_sink, int64_t sink_len, int64_t trips, int kind, double* gops,
                                       double* ms_out, void* stream) {
  if (!dev_sink || sink_len < 256 || sink_len % 256 || sink_len > (1ll << 30) || trips < 1 || !gops ||
      kind < 0 || kind > 2)
    return LBM_IMB_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return LBM_IMB_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return LBM_IMB_ECUDA;
  }
  // exactly the resident blocks (one wave, no tail): at most sink_len threads
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (kind == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbm::fp64_rate_kernel<0>, 256, 0);
  else if (kind == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbm::fp64_rate_kernel<1>, 256, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbm::fp64_rate_kernel<2>, 256, 0);
  long long nb = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  if (nb > sink_len / 256) nb = sink_len / 256;
  const unsigned blocks = (unsigned)nb;
  auto launch = [&]() {
    const double m = 0.9999999999, c = 1e-13;
    if (kind == 0) lbm::fp64_rate_kernel<0><<<blocks, 256, 0, s>>>(dev_sink, (long long)trips, m, c);
    else if (kind == 1) lbm::fp64_rate_kernel<1><<<blocks, 256, 0, s>>>(dev_sink, (long long)trips, m, c);
    else lbm::fp64_rate_kernel<2><<<blocks, 256, 0, s>>>(dev_sink, (long long)trips, m, c);
  };
  launch();  // warm-up
  cudaEventRecord(e0, s);
  launch();
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(ms > 0.f)) return LBM_IMB_ECUDA;
  *gops = (double)blocks * 256.0 * (double)trips * lbm::kFp64Reps * lbm::kFp64Chains / (ms * 1e-3) / 1e9;
  if (ms_out) *ms_out = ms;
  return LBM_IMB_OK;
}
