// K2: fused pull-stream + LBGK collision with the Noble-Torczynski immersed
// moving boundary term (Xiong et al., Eq. 1 with beta of Eq. 2 and the
// Omega^S term), body force F_i = 3 w_i rho (c_i . g_f), and the per-particle
// force/torque sums of Eq. (3), reduced over each warp by owner before one
// FP64 atomic per (warp, particle).
//
// Layout: structure of arrays f[q][z][y][pitch], x fastest; one thread per
// node, one 128-thread CTA per row segment, so the 19 pulled loads of a warp
// are 32 consecutive elements each (shifted by c_x) and the stores are
// aligned.  Opposite directions are processed as pairs: f^eq_{+-} = A +- B
// shares A = w rho (1 - 1.5 u.u + 4.5 (c.u)^2) and B = 3 w rho (c.u).
//
// Storage variants: FP64 (FP64 arithmetic, the parity form); FP32 deviation
// g = f - w rho0 (FP32 arithmetic); FP16 deviation stored as g / w (FP32
// arithmetic).  In the deviation variants the particle-side arithmetic of the
// IMB nodes (solid velocity, per-node force and torque, warp sums) is FP32
// as well, read from a per-particle FP32 kinematics record; the per-particle
// force/torque accumulators are FP64 in every variant.
#include "dev_collide.cuh"

namespace lbm {

template <class LAT, int STORE>
__global__ void __launch_bounds__(128) collide_kernel(View v) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = x < v.nx;
  collide_node<LAT, STORE>(v, active ? x : v.nx - 1, blockIdx.y, blockIdx.z, active);
}

template <class LAT, int STORE>
static void launch_one(const View& v, cudaStream_t s) {
  dim3 grid((v.nx + 127) / 128, v.ny, v.nz);
  collide_kernel<LAT, STORE><<<grid, 128, 0, s>>>(v);
}

void launch_collide(const View& v, cudaStream_t s) {
  if (v.dim == 2) {
    if (v.storage == LBM_IMB_STORE_F64) launch_one<D2Q9, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) launch_one<D2Q9, LBM_IMB_STORE_F32DEV>(v, s);
    else launch_one<D2Q9, LBM_IMB_STORE_F16DEV>(v, s);
  } else {
    if (v.storage == LBM_IMB_STORE_F64) launch_one<D3Q19, LBM_IMB_STORE_F64>(v, s);
    else if (v.storage == LBM_IMB_STORE_F32DEV) launch_one<D3Q19, LBM_IMB_STORE_F32DEV>(v, s);
    else launch_one<D3Q19, LBM_IMB_STORE_F16DEV>(v, s);
  }
}

}  // namespace lbm
