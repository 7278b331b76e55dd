// kernels_params.cu -- per-variable segmented operations around the solver
// that DOGE-Train's pipeline applies between rounds of Alg. 1:
//  * the non-parametric update of eq. 2 (Sec. 3.4),
//    lambda_ij += theta_ij - mean_{k in J_i} theta_ik, and its adjoint;
//  * the output transforms of the parameter predictor (Alg. 3): softmax of
//    alpha-hat over J_i, sigmoid of omega-hat, centring of theta-hat, and
//    their adjoints.
// One thread per variable walks the variable's slots in the fixed order of
// the variable CSR (deterministic).  Padding slots are never touched.
#include "kernels.h"

namespace dg {

__global__ void __launch_bounds__(256) k_nonparam(DevArena A, float* lam, const float* __restrict__ theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  if (e == b) return;
  float s = 0.f;
  for (int k = b; k < e; ++k) s += theta[__ldg(A.var_slots + k)];
  const float mean = s / (float)(e - b);
  for (int k = b; k < e; ++k) {
    const int q = __ldg(A.var_slots + k);
    lam[q] += theta[q] - mean;
  }
}

// out = x - mean over J_i (the centring; its own adjoint)
__global__ void __launch_bounds__(256) k_center(DevArena A, const float* __restrict__ x, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  if (e == b) return;
  float s = 0.f;
  for (int k = b; k < e; ++k) s += x[__ldg(A.var_slots + k)];
  const float mean = s / (float)(e - b);
  for (int k = b; k < e; ++k) {
    const int q = __ldg(A.var_slots + k);
    out[q] = x[q] - mean;
  }
}

__global__ void __launch_bounds__(256) k_param_transform(DevArena A, const float* __restrict__ ah,
                                                          const float* __restrict__ wh,
                                                          const float* __restrict__ th, float* alpha, float* omega,
                                                          float* theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  if (e == b) return;
  if (alpha) {
    float mx = -3.0e38f;
    for (int k = b; k < e; ++k) mx = fmaxf(mx, ah[__ldg(A.var_slots + k)]);
    float z = 0.f;
    for (int k = b; k < e; ++k) z += expf(ah[__ldg(A.var_slots + k)] - mx);
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      alpha[q] = expf(ah[q] - mx) / z;
    }
  }
  if (omega)
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      omega[q] = 1.0f / (1.0f + expf(-wh[q]));
    }
  if (theta) {
    float s = 0.f;
    for (int k = b; k < e; ++k) s += th[__ldg(A.var_slots + k)];
    const float mean = s / (float)(e - b);
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      theta[q] = th[q] - mean;
    }
  }
}

__global__ void __launch_bounds__(256) k_param_transform_bwd(DevArena A, const float* __restrict__ alpha,
                                                              const float* __restrict__ omega,
                                                              const float* __restrict__ ga,
                                                              const float* __restrict__ gw,
                                                              const float* __restrict__ gt, float* gah, float* gwh,
                                                              float* gth) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  if (e == b) return;
  if (gah) {
    float dot = 0.f;
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      dot += alpha[q] * ga[q];
    }
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      gah[q] = alpha[q] * (ga[q] - dot);
    }
  }
  if (gwh)
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      gwh[q] = gw[q] * omega[q] * (1.0f - omega[q]);
    }
  if (gth) {
    float s = 0.f;
    for (int k = b; k < e; ++k) s += gt[__ldg(A.var_slots + k)];
    const float mean = s / (float)(e - b);
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      gth[q] = gt[q] - mean;
    }
  }
}

static unsigned var_blocks(const DevArena& A) { return (unsigned)((A.n + 255) / 256); }

void launch_nonparam(const DevArena& A, float* lam, const float* theta, cudaStream_t st) {
  if (A.n > 0) k_nonparam<<<var_blocks(A), 256, 0, st>>>(A, lam, theta);
}
void launch_center(const DevArena& A, const float* x, float* out, cudaStream_t st) {
  if (A.n > 0) k_center<<<var_blocks(A), 256, 0, st>>>(A, x, out);
}
void launch_param_transform(const DevArena& A, const float* ah, const float* wh, const float* th, float* alpha,
                            float* omega, float* theta, cudaStream_t st) {
  if (A.n > 0) k_param_transform<<<var_blocks(A), 256, 0, st>>>(A, ah, wh, th, alpha, omega, theta);
}
void launch_param_transform_bwd(const DevArena& A, const float* alpha, const float* omega, const float* ga,
                                const float* gw, const float* gt, float* gah, float* gwh, float* gth, cudaStream_t st) {
  if (A.n > 0) k_param_transform_bwd<<<var_blocks(A), 256, 0, st>>>(A, alpha, omega, ga, gw, gt, gah, gwh, gth);
}

}  // namespace dg
