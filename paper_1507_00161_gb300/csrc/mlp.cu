// Learned Davidson preconditioner: a per-element network 4 -> 256 -> 256 -> 256 -> 1
// (ReLU), trained on the GPU by the kernels of this file (not in the paper; the method's
// own Davidson steps provide the training pairs, diagonal Davidson is the fallback).
//
// Parameters (packed, row-major): W1 (256 x 4), b1, W2 (256 x 256), b2, W3 (256 x 256),
// b3, w4 (256), b4 (1).  Activations are row-major (rows = samples).  The dense layers
// run on the library's grouped GEMM: the FP32 network on the split-TF32 tensor-core engine
// (FP32 accuracy), the FP64 one (gradient checks) on the FP64 tiles; everything else in the
// kernels below.
// Loss: mean squared error; optimizer: Adam.
#include <cmath>
#include <type_traits>

#include "common.h"

namespace dmrg {

constexpr int kWd = 256;
constexpr int kIn = 4;

int64_t mlp_n_params() {
  return int64_t(kWd) * kIn + kWd + 2 * (int64_t(kWd) * kWd + kWd) + kWd + 1;
}

template <class T>
struct MlpOffsets {
  int64_t W1, b1, W2, b2, W3, b3, w4, b4;
  MlpOffsets() {
    W1 = 0;
    b1 = W1 + int64_t(kWd) * kIn;
    W2 = b1 + kWd;
    b2 = W2 + int64_t(kWd) * kWd;
    W3 = b2 + kWd;
    b3 = W3 + int64_t(kWd) * kWd;
    w4 = b3 + kWd;
    b4 = w4 + kWd;
  }
};

// ------------------------------------------------------------------------------------
// elementwise kernels
// ------------------------------------------------------------------------------------
template <class T>
__global__ void k_bias_relu(T* __restrict__ Z, const T* __restrict__ b, T* __restrict__ H,
                            int64_t rows, int cols) {
  const int64_t n = rows * cols;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const T z = Z[i] + b[i % cols];
    Z[i] = z;
    H[i] = z > T(0) ? z : T(0);
  }
}

template <class T>
__global__ void k_add_scalar(T* __restrict__ y, const T* __restrict__ b, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] += b[0];
}

// dZ = dH * (Z > 0)
template <class T>
__global__ void k_relu_grad(const T* __restrict__ Z, T* __restrict__ dH, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    if (!(Z[i] > T(0))) dH[i] = T(0);
}

// column sums of a rows x cols matrix (one thread per column, fixed order)
template <class T>
__global__ void k_colsum(const T* __restrict__ A, int64_t rows, int cols, T* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  T s = T(0);
  for (int64_t r = 0; r < rows; ++r) s += A[r * cols + c];
  out[c] = s;
}

// dY = 2 (Y - T) / B ; per-block partial sums of (Y - T)^2
template <class T>
__global__ void k_mse(const T* __restrict__ Y, const T* __restrict__ Tg, int64_t B,
                      T* __restrict__ dY, double* __restrict__ part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < B;
       i += int64_t(gridDim.x) * blockDim.x) {
    const T d = Y[i] - Tg[i];
    dY[i] = T(2) * d / T(B);
    s += double(d) * double(d);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (int(threadIdx.x) < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

template <class T>
__global__ void k_adam(T* __restrict__ p, const T* __restrict__ g, T* __restrict__ m,
                       T* __restrict__ v, int64_t n, double lr, double b1, double b2, double eps,
                       double c1, double c2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const double gi = double(g[i]);
    const double mi = b1 * double(m[i]) + (1.0 - b1) * gi;
    const double vi = b2 * double(v[i]) + (1.0 - b2) * gi * gi;
    m[i] = T(mi);
    v[i] = T(vi);
    p[i] = T(double(p[i]) - lr * (mi / c1) / (sqrt(vi / c2) + eps));
  }
}

// gather rows of a sample table into a minibatch (samples: n_in features + target)
template <class T>
__global__ void k_gather(const T* __restrict__ S, const int32_t* __restrict__ idx, int64_t B,
                         T* __restrict__ X, T* __restrict__ Tg) {
  for (int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; b < B;
       b += int64_t(gridDim.x) * blockDim.x) {
    const T* s = S + int64_t(idx[b]) * (kIn + 1);
#pragma unroll
    for (int j = 0; j < kIn; ++j) X[b * kIn + j] = s[j];
    Tg[b] = s[kIn];
  }
}

// features of every element of a Davidson iterate:
//   asinh(theta - D_i), r_i sqrt(n)/|r|, x_i sqrt(n), d_i sqrt(n)/|d|,  d_i = r_i/(theta - D_i)
// (the clamped diagonal correction); sc = {theta, |r|^2, |d|^2}
// features and targets are O(1) by construction; bound the rare outliers (an element whose
// diagonal sits on theta, a residual at rounding level) so that FP32 training stays finite
__device__ __forceinline__ float clampf(double v) {
  return float(v != v ? 0.0 : fmin(fmax(v, -1e4), 1e4));
}

template <class T>
__global__ void k_features(const double* __restrict__ r, const double* __restrict__ x,
                           const double* __restrict__ diag, const double* __restrict__ sc,
                           int64_t n, T* __restrict__ X) {
  const double th = sc[0];
  const double sn = sqrt(double(n));
  const double ir = sc[1] > 0 ? sn / sqrt(sc[1]) : 0.0;
  const double id = sc[2] > 0 ? sn / sqrt(sc[2]) : 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    double den = th - diag[i];
    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
    X[i * kIn + 0] = T(clampf(asinh(th - diag[i])));
    X[i * kIn + 1] = T(clampf(r[i] * ir));
    X[i * kIn + 2] = T(clampf(x[i] * sn));
    X[i * kIn + 3] = T(clampf(r[i] / den * id));
  }
}

// training pairs from one saved iterate: features of sampled elements and the target
// e_i sqrt(n)/|e|, e = psi - x (x . psi) with the sign of psi making x . psi >= 0;
// sc = {theta, |r|^2, |d|^2, x.psi, |e|^2}; elements i = start + k stride
__global__ void k_harvest(const double* __restrict__ r, const double* __restrict__ x,
                          const double* __restrict__ psi, const double* __restrict__ diag,
                          const double* __restrict__ sc, int64_t n, int64_t start, int64_t stride,
                          int64_t count, float* __restrict__ out) {
  const double th = sc[0];
  const double sn = sqrt(double(n));
  const double ir = sc[1] > 0 ? sn / sqrt(sc[1]) : 0.0;
  const double id = sc[2] > 0 ? sn / sqrt(sc[2]) : 0.0;
  const double ov = sc[3];
  const double sg = ov < 0 ? -1.0 : 1.0;
  // an iterate that already equals the eigenvector (|e| at rounding level) has no error
  // direction to learn: its targets are zero
  const double ie = sc[4] > 1e-20 ? sn / sqrt(sc[4]) : 0.0;
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < count;
       k += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = start + k * stride;
    double den = th - diag[i];
    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
    float* o = out + k * (kIn + 1);
    o[0] = clampf(asinh(th - diag[i]));
    o[1] = clampf(r[i] * ir);
    o[2] = clampf(x[i] * sn);
    o[3] = clampf(r[i] / den * id);
    o[4] = clampf(sg * (psi[i] - x[i] * ov) * ie);
  }
}

// e = psi - x (x . psi) (sign of psi as above) for |e|^2
__global__ void k_err_vec(const double* __restrict__ x, const double* __restrict__ psi,
                          const double* __restrict__ sc, int64_t n, double* __restrict__ e) {
  const double ov = sc[3];
  const double sg = ov < 0 ? -1.0 : 1.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    e[i] = sg * (psi[i] - x[i] * ov);
}

// out_double[i] = y[i]
template <class T>
__global__ void k_to_double(const T* __restrict__ y, double* __restrict__ out, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] = double(y[i]);
}

static int grid_for(int64_t n) {
  return int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
}

// C (M x N, ldc) = op(A) op(B) through the task-list GEMM; sizes of the three buffers in
// elements for the host-side range check
template <class T>
static void gemm(T* C, int ldc, const T* A, int lda, bool ta, const T* B, int ldb, bool tb, int M,
                 int N, int K, int64_t nA, int64_t nB, int64_t nC, cudaStream_t s) {
  TaskList L;
  L.begin_task(Operand{0, B_Y, ldc}, M, N);
  L.add_term(Operand{0, B_X, lda}, Operand{0, B_U, ldb}, K, (ta ? 1 : 0) | (tb ? 2 : 0), 1.0);
  int64_t be[NBASE] = {0};
  be[B_X] = nA;
  be[B_U] = nB;
  be[B_Y] = nC;
  DevTaskList d;
  if constexpr (std::is_same<T, float>::value) {
    d.build(L, be, s, 0);   // every task in 64 x 64 tensor-core tiles
    Bases<void> b{};
    b.p[B_X] = const_cast<T*>(A);
    b.p[B_U] = const_cast<T*>(B);
    b.p[B_Y] = C;
    run_gemm_tasks_tc<float, float, float>(d, b, 1, s);
  } else {
    d.build(L, be, s);
    Bases<T> b{};
    b.p[B_X] = const_cast<T*>(A);
    b.p[B_U] = const_cast<T*>(B);
    b.p[B_Y] = C;
    run_gemm_tasks<T>(d, b, 1, s);
  }
  DMRG_CUDA(cudaStreamSynchronize(s));   // the list buffers are released on return
}

template <class T>
void mlp_forward(const T* P, const T* X, int64_t B, MlpActs<T>& a, cudaStream_t s) {
  MlpOffsets<T> o;
  const int64_t np = mlp_n_params();
  a.ensure(B);
  const int64_t nh = B * kWd;
  gemm<T>(a.Z1.p, kWd, X, kIn, false, P + o.W1, kIn, true, int(B), kWd, kIn, B * kIn, np - o.W1,
          nh, s);
  k_bias_relu<T><<<grid_for(nh), 256, 0, s>>>(a.Z1.p, P + o.b1, a.H1.p, B, kWd);
  DMRG_LAUNCHED();
  gemm<T>(a.Z2.p, kWd, a.H1.p, kWd, false, P + o.W2, kWd, true, int(B), kWd, kWd, nh, np - o.W2,
          nh, s);
  k_bias_relu<T><<<grid_for(nh), 256, 0, s>>>(a.Z2.p, P + o.b2, a.H2.p, B, kWd);
  DMRG_LAUNCHED();
  gemm<T>(a.Z3.p, kWd, a.H2.p, kWd, false, P + o.W3, kWd, true, int(B), kWd, kWd, nh, np - o.W3,
          nh, s);
  k_bias_relu<T><<<grid_for(nh), 256, 0, s>>>(a.Z3.p, P + o.b3, a.H3.p, B, kWd);
  DMRG_LAUNCHED();
  gemm<T>(a.Y.p, 1, a.H3.p, kWd, false, P + o.w4, kWd, true, int(B), 1, kWd, nh, np - o.w4, B, s);
  k_add_scalar<T><<<grid_for(B), 256, 0, s>>>(a.Y.p, P + o.b4, B);
  DMRG_LAUNCHED();
}

// loss (mean squared error) and gradient G of the parameters; forward must have run on X
template <class T>
double mlp_backward(const T* P, const T* X, const T* Tg, int64_t B, MlpActs<T>& a, T* G,
                    cudaStream_t s) {
  MlpOffsets<T> o;
  const int64_t np = mlp_n_params();
  const int64_t nh = B * kWd;
  const int nb = 64;
  a.part.alloc(nb);
  k_mse<T><<<nb, 256, 0, s>>>(a.Y.p, Tg, B, a.dY.p, a.part.p);
  DMRG_LAUNCHED();
  // output layer
  gemm<T>(G + o.w4, kWd, a.dY.p, 1, true, a.H3.p, kWd, false, 1, kWd, int(B), B, nh, np - o.w4, s);
  k_colsum<T><<<1, 32, 0, s>>>(a.dY.p, B, 1, G + o.b4);
  DMRG_LAUNCHED();
  gemm<T>(a.dH.p, kWd, a.dY.p, 1, false, P + o.w4, kWd, false, int(B), kWd, 1, B, np - o.w4, nh, s);
  // layer 3
  k_relu_grad<T><<<grid_for(nh), 256, 0, s>>>(a.Z3.p, a.dH.p, nh);
  DMRG_LAUNCHED();
  gemm<T>(G + o.W3, kWd, a.dH.p, kWd, true, a.H2.p, kWd, false, kWd, kWd, int(B), nh, nh,
          np - o.W3, s);
  k_colsum<T><<<1, kWd, 0, s>>>(a.dH.p, B, kWd, G + o.b3);
  DMRG_LAUNCHED();
  gemm<T>(a.dZ.p, kWd, a.dH.p, kWd, false, P + o.W3, kWd, false, int(B), kWd, kWd, nh, np - o.W3,
          nh, s);
  // layer 2
  k_relu_grad<T><<<grid_for(nh), 256, 0, s>>>(a.Z2.p, a.dZ.p, nh);
  DMRG_LAUNCHED();
  gemm<T>(G + o.W2, kWd, a.dZ.p, kWd, true, a.H1.p, kWd, false, kWd, kWd, int(B), nh, nh,
          np - o.W2, s);
  k_colsum<T><<<1, kWd, 0, s>>>(a.dZ.p, B, kWd, G + o.b2);
  DMRG_LAUNCHED();
  gemm<T>(a.dH.p, kWd, a.dZ.p, kWd, false, P + o.W2, kWd, false, int(B), kWd, kWd, nh, np - o.W2,
          nh, s);
  // layer 1
  k_relu_grad<T><<<grid_for(nh), 256, 0, s>>>(a.Z1.p, a.dH.p, nh);
  DMRG_LAUNCHED();
  gemm<T>(G + o.W1, kIn, a.dH.p, kWd, true, X, kIn, false, kWd, kIn, int(B), nh, B * kIn,
          np - o.W1, s);
  k_colsum<T><<<1, kWd, 0, s>>>(a.dH.p, B, kWd, G + o.b1);
  DMRG_LAUNCHED();
  std::vector<double> part(nb);
  DMRG_CUDA(cudaMemcpyAsync(part.data(), a.part.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
  DMRG_CUDA(cudaStreamSynchronize(s));
  double loss = 0.0;
  for (double x : part) loss += x;
  return loss / double(B);
}

template <class T>
void mlp_adam(T* P, const T* G, T* m, T* v, int64_t n, double lr, int step, cudaStream_t s) {
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double c1 = 1.0 - std::pow(b1, step), c2 = 1.0 - std::pow(b2, step);
  k_adam<T><<<grid_for(n), 256, 0, s>>>(P, G, m, v, n, lr, b1, b2, eps, c1, c2);
  DMRG_LAUNCHED();
}

template <class T>
void mlp_gather(const T* S, const int32_t* idx, int64_t B, T* X, T* Tg, cudaStream_t s) {
  k_gather<T><<<grid_for(B), 256, 0, s>>>(S, idx, B, X, Tg);
  DMRG_LAUNCHED();
}

template <class T>
void mlp_features(const double* r, const double* x, const double* diag, const double* sc,
                  int64_t n, T* X, cudaStream_t s) {
  k_features<T><<<grid_for(n), 256, 0, s>>>(r, x, diag, sc, n, X);
  DMRG_LAUNCHED();
}

template <class T>
void mlp_output_to_double(const T* y, double* out, int64_t n, cudaStream_t s) {
  k_to_double<T><<<grid_for(n), 256, 0, s>>>(y, out, n);
  DMRG_LAUNCHED();
}

void mlp_harvest(const double* r, const double* x, const double* psi, const double* diag,
                 const double* sc, int64_t n, int64_t start, int64_t stride, int64_t count,
                 float* out, cudaStream_t s) {
  if (count <= 0) return;
  k_harvest<<<grid_for(count), 256, 0, s>>>(r, x, psi, diag, sc, n, start, stride, count, out);
  DMRG_LAUNCHED();
}

void mlp_err_vec(const double* x, const double* psi, const double* sc, int64_t n, double* e,
                 cudaStream_t s) {
  k_err_vec<<<grid_for(n), 256, 0, s>>>(x, psi, sc, n, e);
  DMRG_LAUNCHED();
}

template void mlp_forward<float>(const float*, const float*, int64_t, MlpActs<float>&, cudaStream_t);
template void mlp_forward<double>(const double*, const double*, int64_t, MlpActs<double>&,
                                  cudaStream_t);
template double mlp_backward<float>(const float*, const float*, const float*, int64_t,
                                    MlpActs<float>&, float*, cudaStream_t);
template double mlp_backward<double>(const double*, const double*, const double*, int64_t,
                                     MlpActs<double>&, double*, cudaStream_t);
template void mlp_adam<float>(float*, const float*, float*, float*, int64_t, double, int,
                              cudaStream_t);
template void mlp_gather<float>(const float*, const int32_t*, int64_t, float*, float*, cudaStream_t);
template void mlp_features<float>(const double*, const double*, const double*, const double*,
                                  int64_t, float*, cudaStream_t);
template void mlp_output_to_double<float>(const float*, double*, int64_t, cudaStream_t);

}  // namespace dmrg
