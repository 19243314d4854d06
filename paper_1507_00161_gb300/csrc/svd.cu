// Eigendecomposition of the reduced density matrices of the truncation (the basis change
// "by the SVD theorem" of the two-site step):
//     rho_Q = B B^T,   B = the wave-function block of sector Q (d x e; its transpose when
//                      the right block is truncated; [psi_0 psi_1] / sqrt(2) when two
//                      states are targeted),
// computed from the singular value decomposition of B by one-sided Jacobi (Hestenes)
// rotations in FP64:
//   - d > E (E = columns of B): A = B (d x E); rotating column pairs of A until they are
//     mutually orthogonal gives A = U Sigma, so the eigenvectors of rho are the normalised
//     columns, the eigenvalues their squared norms, and the remaining d - E eigenvalues
//     are exactly zero;
//   - d <= E: A = B^T (E x d) and the rotations are accumulated in V (d x d), A V = W with
//     orthogonal columns, so rho = V W^T W V^T: eigenvectors = columns of V, eigenvalues
//     = squared column norms of W.
// The problem is min(d, E) columns instead of the d x d two-sided problem, and singular
// values come out with high relative accuracy.
//
// A sector is processed by a thread-block cluster of C CTAs (C = 1, 8 or 16).  CTA k holds
// rows [k R, (k + 1) R) of A (and of V) in its shared memory, so a column rotation only
// touches local rows.  Each round of the round-robin ordering (m/2 disjoint column pairs):
//   1. every CTA sums alpha = |a_p|^2, beta = |a_q|^2, gamma = a_p . a_q over its rows;
//   2. cluster barrier; every CTA adds the C partial sums of every pair in rank order
//      (distributed shared memory), so all CTAs derive the same rotation
//        zeta = (beta - alpha) / (2 gamma), t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//        c = 1 / sqrt(1 + t^2), s = c t,   a_p <- c a_p - s a_q,  a_q <- s a_p + c a_q
//      (skipped when |gamma| <= tol sqrt(alpha beta));
//   3. every CTA rotates its rows.
// Partial sums are double-buffered, so one cluster barrier per round suffices.  A sweep
// without a rotation ends the iteration (every CTA takes the same decision); after
// kMaxSweeps sweeps the job raises the context's non-convergence flag and still writes
// its result.  Output per sector: eigenvalues descending (ties by column index) at w_off,
// the eigenvectors as the columns of a d x d row-major matrix at vs_off, each with its
// largest |component| positive (lowest row on ties).  Deterministic: fixed reduction
// orders everywhere, no atomics on floating point.
#include <cooperative_groups.h>
#include <stdint.h>

#include <mutex>

#include "common.h"

namespace cg = cooperative_groups;

namespace dmrg {

namespace {

constexpr int kMaxSweeps = 40;
constexpr size_t kSvdSmemMax = 226 * 1024;   // dynamic share; the static part needs a little

struct SvdShape {
  int d, E, rows, cols, needV, R, Rv, P;
};

__device__ __forceinline__ SvdShape svd_shape(const SvdJob& j, int C) {
  SvdShape s;
  s.d = j.D;
  s.E = j.e * j.roots;
  s.needV = s.d < s.E;
  s.cols = s.needV ? s.d : s.E;
  s.rows = s.needV ? s.E : s.d;
  s.R = (s.rows + C - 1) / C;
  s.Rv = s.needV ? (s.d + C - 1) / C : 0;
  s.P = (s.cols + 1) / 2;
  return s;
}

// element (i, j) of B (d x E)
__device__ __forceinline__ double b_at(const SvdJob& jb, const double* __restrict__ psi0,
                                       const double* __restrict__ psi1, int i, int j) {
  const double* src = psi0;
  double sc = 1.0;
  if (j >= jb.e) {
    src = psi1;
    j -= jb.e;
  }
  if (jb.roots == 2) sc = 0.70710678118654752440;
  const int64_t o = jb.trans ? jb.src + int64_t(j) * jb.D + i : jb.src + int64_t(i) * jb.e + j;
  return sc * src[o];
}

__device__ __forceinline__ void round_pair(int m, int r, int k, int& p, int& q) {
  int a, b;
  if (k == 0) {
    a = m - 1;
    b = r;
  } else {
    a = (r + k) % (m - 1);
    b = (r - k + (m - 1)) % (m - 1);
  }
  p = min(a, b);
  q = max(a, b);
}

// NT threads per CTA (256; 64 for single-CTA sectors was measured slower: their rounds are
// latency-bound, and fewer threads lengthen each round more than the shorter barriers save)
template <int NT>
__global__ void __launch_bounds__(NT, 1)
    k_svd_jacobi(const SvdJob* __restrict__ jobs, const double* __restrict__ psi0,
                 const double* __restrict__ psi1, double* __restrict__ w_out,
                 double* __restrict__ vs_out, int* __restrict__ noconv, double tol_scale) {
  extern __shared__ __align__(16) double svd_sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = int(cl.num_blocks());
  const int rank = int(cl.block_rank());
  const SvdJob jb = jobs[blockIdx.x / C];
  const SvdShape S = svd_shape(jb, C);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = NT / 32;
  const int ld = S.cols + 1;   // odd leading dimension: fewer bank conflicts across rows
  // shared layout: A rows, V rows, partials [2][3 P] (also used for final norms and signs),
  // rotations [2 P], pair indices
  double* A = svd_sm;
  double* V = A + size_t(S.R) * ld;
  double* part = V + size_t(S.Rv) * ld;
  const int partN = max(3 * S.P, 2 * S.cols + 2);
  double* rot = part + 2 * partN;
  int* pq = reinterpret_cast<int*>(rot + 2 * S.P);
  __shared__ int s_flag;

  const int r0 = rank * S.R, r1 = min(S.rows, r0 + S.R);
  const int nr = max(0, r1 - r0);
  const int v0 = rank * S.Rv, v1 = min(S.d, v0 + S.Rv);
  const int nv = max(0, v1 - v0);
  for (int e = tid; e < nr * S.cols; e += NT) {
    const int r = e / S.cols, c = e - r * S.cols;
    A[r * ld + c] = S.needV ? b_at(jb, psi0, psi1, c, r0 + r) : b_at(jb, psi0, psi1, r0 + r, c);
  }
  for (int e = tid; e < nv * S.cols; e += NT) {
    const int r = e / S.cols, c = e - r * S.cols;
    V[r * ld + c] = (v0 + r == c) ? 1.0 : 0.0;
  }
  const int m = S.cols + (S.cols & 1);
  const double tol = tol_scale * sqrt(double(max(S.rows, 1)));
  int sweep = 0;
  bool converged = S.cols <= 1;
  int buf = 0;
  cl.sync();
  while (!converged && sweep < kMaxSweeps) {
    if (tid == 0) s_flag = 0;
    for (int r = 0; r < m - 1; ++r) {
      // 1. partial sums over local rows, one warp per pair
      double* pb = part + buf * partN;
      for (int k = warp; k < m / 2; k += nwarp) {
        int p, q;
        round_pair(m, r, k, p, q);
        double al = 0.0, be = 0.0, ga = 0.0;
        if (q < S.cols)
          for (int i = lane; i < nr; i += 32) {
            const double x = A[i * ld + p], y = A[i * ld + q];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_down_sync(0xffffffffu, al, o);
          be += __shfl_down_sync(0xffffffffu, be, o);
          ga += __shfl_down_sync(0xffffffffu, ga, o);
        }
        if (lane == 0) {
          pb[3 * k] = al;
          pb[3 * k + 1] = be;
          pb[3 * k + 2] = ga;
        }
      }
      cl.sync();
      // 2. cluster sums in rank order and the rotations (identical in every CTA)
      for (int k = tid; k < m / 2; k += NT) {
        int p, q;
        round_pair(m, r, k, p, q);
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int c = 0; c < C; ++c) {
          const double* rp = cl.map_shared_rank(pb, c);
          al += rp[3 * k];
          be += rp[3 * k + 1];
          ga += rp[3 * k + 2];
        }
        double cs = 1.0, sn = 0.0;
        if (q < S.cols && al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          cs = 1.0 / sqrt(1.0 + t * t);
          sn = cs * t;
          s_flag = 1;
        }
        rot[2 * k] = cs;
        rot[2 * k + 1] = sn;
        pq[2 * k] = p;
        pq[2 * k + 1] = q;
      }
      __syncthreads();
      // 3. rotate the local rows of A and V
      const int half = m / 2;
      for (int e = tid; e < half * nr; e += NT) {
        const int k = e / nr, i = e - k * nr;
        const double sn = rot[2 * k + 1];
        if (sn == 0.0) continue;
        const double cs = rot[2 * k];
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const double x = A[i * ld + p], y = A[i * ld + q];
        A[i * ld + p] = cs * x - sn * y;
        A[i * ld + q] = sn * x + cs * y;
      }
      for (int e = tid; e < half * nv; e += NT) {
        const int k = e / nv, i = e - k * nv;
        const double sn = rot[2 * k + 1];
        if (sn == 0.0) continue;
        const double cs = rot[2 * k];
        const int p = pq[2 * k], q = pq[2 * k + 1];
        const double x = V[i * ld + p], y = V[i * ld + q];
        V[i * ld + p] = cs * x - sn * y;
        V[i * ld + q] = sn * x + cs * y;
      }
      __syncthreads();
      buf ^= 1;
    }
    ++sweep;
    converged = s_flag == 0;
    __syncthreads();
  }
  if (!converged && rank == 0 && tid == 0) atomicExch(noconv, 1);

  // final squared column norms (cluster sums in rank order)
  double* pb = part + buf * partN;
  for (int c = warp; c < S.cols; c += nwarp) {
    double al = 0.0;
    for (int i = lane; i < nr; i += 32) al = fma(A[i * ld + c], A[i * ld + c], al);
    for (int o = 16; o > 0; o >>= 1) al += __shfl_down_sync(0xffffffffu, al, o);
    if (lane == 0) pb[c] = al;
  }
  cl.sync();
  double* nrm = rot;   // reuse: cols norms (rot holds 2 P >= cols entries)
  for (int c = tid; c < S.cols; c += NT) {
    double al = 0.0;
    for (int k = 0; k < C; ++k) al += cl.map_shared_rank(pb, k)[c];
    nrm[c] = al;
  }
  __syncthreads();
  // rank of each column: descending weight, ties by index
  int* order = pq;   // order[c] = output position of column c
  for (int c = tid; c < S.cols; c += NT) {
    const double wc = nrm[c];
    int pos = 0;
    for (int j = 0; j < S.cols; ++j) {
      const double wj = nrm[j];
      if (wj > wc || (wj == wc && j < c)) ++pos;
    }
    order[c] = pos;
  }
  __syncthreads();
  // sign of every eigenvector: its largest |component| (lowest row on ties) positive.
  // Local candidates (value, row) in the other partial buffer, then a rank-order merge.
  const double* U = S.needV ? V : A;
  const int nu = S.needV ? nv : nr;
  const int u0 = S.needV ? v0 : r0;
  double* pc = part + (buf ^ 1) * partN;
  for (int c = warp; c < S.cols; c += nwarp) {
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int i = lane; i < nu; i += 32) {
      const double a = fabs(U[i * ld + c]);
      if (a > bv) {
        bv = a;
        bi = u0 + i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      pc[2 * c] = bv;
      pc[2 * c + 1] = double(bi);
    }
  }
  cl.sync();
  double* sgn = pb;   // own norms buffer is no longer read by anyone after the next barrier
  __syncthreads();
  for (int c = tid; c < S.cols; c += NT) {
    double bv = -1.0, bi = 1e300;
    for (int k = 0; k < C; ++k) {
      const double* rp = cl.map_shared_rank(pc, k);
      if (rp[2 * c] > bv || (rp[2 * c] == bv && rp[2 * c + 1] < bi)) {
        bv = rp[2 * c];
        bi = rp[2 * c + 1];
      }
    }
    // the owner of row bi holds the component's sign; fetch it
    const int row = int(bi);
    double val = 1.0;
    if (row >= 0 && row < (S.needV ? S.d : S.rows)) {
      const int owner = row / (S.needV ? S.Rv : S.R);
      const double* ru = S.needV ? V : A;
      const double* remote = cl.map_shared_rank(ru, owner);
      val = remote[(row - owner * (S.needV ? S.Rv : S.R)) * ld + c];
    }
    sgn[2 * c] = val < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  // outputs: eigenvalues (rank 0) and the eigenvector rows this CTA holds
  if (rank == 0)
    for (int c = tid; c < S.d; c += NT)
      w_out[jb.w_off + c] = 0.0;
  __syncthreads();
  if (rank == 0)
    for (int c = tid; c < S.cols; c += NT) w_out[jb.w_off + order[c]] = nrm[c];
  for (int e = tid; e < nu * S.d; e += NT) {
    const int i = e / S.d, c = e - i * S.d;   // row i of U (global row u0 + i), output column c
    vs_out[jb.vs_off + int64_t(u0 + i) * S.d + c] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < nu * S.cols; e += NT) {
    const int i = e / S.cols, c = e - i * S.cols;
    double v = U[i * ld + c] * sgn[2 * c];
    if (!S.needV) v = nrm[c] > 0.0 ? v / sqrt(nrm[c]) : 0.0;
    vs_out[jb.vs_off + int64_t(u0 + i) * S.d + order[c]] = v;
  }
  // no CTA may leave while others still read its shared memory
  cl.sync();
}

}  // namespace

size_t svd_smem_limit() { return kSvdSmemMax; }

size_t svd_smem_bytes(const SvdJob& j, int C) {
  const int d = j.D, E = j.e * j.roots;
  const int needV = d < E;
  const int cols = needV ? d : E, rows = needV ? E : d;
  const int R = (rows + C - 1) / C, Rv = needV ? (d + C - 1) / C : 0, P = (cols + 1) / 2;
  const int ld = cols + 1;
  const int partN = std::max(3 * P, 2 * cols + 2);
  return sizeof(double) * (size_t(R + Rv) * ld + 2 * size_t(partN) + 2 * size_t(P)) +
         sizeof(int) * 2 * size_t(P) + 16;
}

void svd_jacobi(const SvdJob* d_jobs, int n_jobs, int C, size_t smem, const double* psi0,
                const double* psi1, double* w, double* vs, int* d_noconv, cudaStream_t s) {
  if (n_jobs <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    DMRG_CUDA(cudaFuncSetAttribute(k_svd_jacobi<256>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSvdSmemMax)));
    DMRG_CUDA(cudaFuncSetAttribute(k_svd_jacobi<256>,
                                   cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  });
  DMRG_REQUIRE(smem <= kSvdSmemMax, DMRG_EINVAL, "internal: SVD job exceeds shared memory");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(n_jobs) * unsigned(C), 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(C);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  DMRG_CUDA(cudaLaunchKernelEx(&cfg, k_svd_jacobi<256>, d_jobs, psi0, psi1, w, vs, d_noconv,
                               2.220446049250313e-16));
  DMRG_LAUNCHED();
}

}  // namespace dmrg
