// CUDA kernels of the DMRG hot path (sm_103a).
//
//  * task-list GEMMs: C (M x N) (+)= sum_t alpha_t op(A_t) op(B_t) over thousands of small
//    per-sector blocks (superblock product, reduced density matrices, renormalization,
//    wave-function transformation).  Tiny tasks run one per warp straight from L1/L2;
//    large tasks are cut into 64 x 64 tiles staged through shared memory.
//  * copy tasks: scaled sums of operator blocks into enlarged-operator sub-blocks.
//  * Davidson vector kernels with deterministic (fixed-order) reductions.
//  * symmetric eigensolver: parallel-ordered cyclic Jacobi, one thread block per matrix,
//    FP64 (reduced density matrices per sector and the small Ritz problem).
//  * selection of the M-th largest weight (bitonic sort in one block) and kept counts.
#include <cuda_runtime.h>
#include <math.h>

#include <atomic>
#include <mutex>

#include "common.h"

namespace dmrg {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_upload_bytes{0}, g_upload_ns{0};
std::atomic<int64_t> g_malloc_count{0}, g_malloc_ns{0};

constexpr int kWarp = 32;

// ------------------------------------------------------------------------------------
// task-list GEMM, one warp per task
// ------------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T ld_op(const T* base, int trans, int ld, int r, int c) {
  // logical element (r, c) of op(X)
  return trans ? base[(int64_t)c * ld + r] : base[(int64_t)r * ld + c];
}

template <class T>
__global__ void __launch_bounds__(256) k_gemm_small(const GemmTask* __restrict__ tasks,
                                                    int64_t n_tasks,
                                                    const GemmTerm* __restrict__ terms,
                                                    Bases<T> b, int beta_zero,
                                                    const int32_t* __restrict__ active) {
  if (active && !active[0]) return;
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / kWarp;
  int lane = threadIdx.x & (kWarp - 1);
  if (w >= n_tasks) return;
  const GemmTask t = tasks[w];
  T* C = b.p[t.C.base] + t.C.off;
  const int MN = t.M * t.N;
  for (int idx = lane; idx < MN; idx += kWarp) {
    const int m = idx / t.N, n = idx - m * t.N;
    T acc = T(0);
    for (int j = t.t0; j < t.t1; ++j) {
      const GemmTerm g = terms[j];
      const T* A = b.p[g.A.base] + g.A.off;
      const T* B = b.p[g.B.base] + g.B.off;
      const int ta = g.trans & 1, tb = (g.trans >> 1) & 1;
      T s = T(0);
      for (int k = 0; k < g.K; ++k)
        s = fma(ld_op(A, ta, g.A.ld, m, k), ld_op(B, tb, g.B.ld, k, n), s);
      acc = fma(T(g.alpha), s, acc);
    }
    T* c = C + (int64_t)m * t.C.ld + n;
    *c = beta_zero ? acc : (*c + acc);
  }
}

// ------------------------------------------------------------------------------------
// task-list GEMM, 64 x 64 tiles, 256 threads (16 x 16, 4 x 4 outputs each)
// ------------------------------------------------------------------------------------
constexpr int TM = 64, TN = 64, TK = 16;

template <class T>
__global__ void __launch_bounds__(256) k_gemm_tiled(const GemmTile* __restrict__ tiles,
                                                    const GemmTask* __restrict__ tasks,
                                                    const GemmTerm* __restrict__ terms,
                                                    Bases<T> b, int beta_zero,
                                                    const int32_t* __restrict__ active) {
  if (active && !active[0]) return;
  __shared__ T As[TK][TM + 1];
  __shared__ T Bs[TK][TN + 1];
  const GemmTile tl = tiles[blockIdx.x];
  const GemmTask t = tasks[tl.task];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int jt = t.t0; jt < t.t1; ++jt) {
    const GemmTerm g = terms[jt];
    const T* A = b.p[g.A.base] + g.A.off;
    const T* B = b.p[g.B.base] + g.B.off;
    const int ta = g.trans & 1, tb = (g.trans >> 1) & 1;
    const T alpha = T(g.alpha);
    for (int k0 = 0; k0 < g.K; k0 += TK) {
      for (int e = threadIdx.x; e < TK * TM; e += 256) {
        int kk = e / TM, mm = e - kk * TM;
        int gm = tl.m0 + mm, gk = k0 + kk;
        As[kk][mm] = (gm < t.M && gk < g.K) ? alpha * ld_op(A, ta, g.A.ld, gm, gk) : T(0);
      }
      for (int e = threadIdx.x; e < TK * TN; e += 256) {
        int kk = e / TN, nn = e - kk * TN;
        int gn = tl.n0 + nn, gk = k0 + kk;
        Bs[kk][nn] = (gn < t.N && gk < g.K) ? ld_op(B, tb, g.B.ld, gk, gn) : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  T* C = b.p[t.C.base] + t.C.off;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = tl.m0 + ty + 16 * i;
    if (gm >= t.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = tl.n0 + tx + 16 * j;
      if (gn >= t.N) continue;
      T* c = C + (int64_t)gm * t.C.ld + gn;
      *c = beta_zero ? acc[i][j] : (*c + acc[i][j]);
    }
  }
}


static void check_range(const Operand& o, int rows, int cols, const int64_t* be,
                        const char* what) {
  if (rows <= 0 || cols <= 0) return;
  DMRG_REQUIRE(o.base >= 0 && o.base < NBASE && be[o.base] > 0, DMRG_EINVAL,
               std::string("internal: task operand on an unset base (") + what + ")");
  DMRG_REQUIRE(o.ld >= cols && o.off >= 0, DMRG_EINVAL,
               std::string("internal: bad leading dimension (") + what + ")");
  int64_t last = o.off + int64_t(rows - 1) * o.ld + (cols - 1);
  DMRG_REQUIRE(last < be[o.base], DMRG_EINVAL,
               std::string("internal: task operand out of range (") + what + ")");
}

void validate_copy_tasks(const CopyList& L, const int64_t* be) {
  for (const auto& t : L.tasks) {
    check_range(t.dst, t.rows, t.cols, be, "copy dst");
    for (int j = t.t0; j < t.t1; ++j) check_range(L.terms[j].src, t.rows, t.cols, be, "copy src");
  }
}

void DevTaskList::build(const TaskList& L, const int64_t* be, cudaStream_t s,
                        int64_t small_limit) {
  for (const auto& t : L.tasks) {
    check_range(t.C, t.M, t.N, be, "C");
    for (int j = t.t0; j < t.t1; ++j) {
      const GemmTerm& g = L.terms[j];
      if (g.K <= 0) continue;
      if (g.trans & 1) check_range(g.A, g.K, t.M, be, "A^T");
      else check_range(g.A, t.M, g.K, be, "A");
      if (g.trans & 2) check_range(g.B, t.N, g.K, be, "B^T");
      else check_range(g.B, g.K, t.N, be, "B");
    }
  }
  std::vector<GemmTask> sm, lg;
  std::vector<GemmTile> tl;
  flops = 0;
  for (const auto& t : L.tasks) {
    for (int j = t.t0; j < t.t1; ++j) flops += 2.0 * t.M * t.N * double(L.terms[j].K);
    if (t.M <= 0 || t.N <= 0) continue;
    if (int64_t(t.M) * t.N <= small_limit) {
      sm.push_back(t);
    } else {
      int id = int(lg.size());
      lg.push_back(t);
      for (int m0 = 0; m0 < t.M; m0 += TM)
        for (int n0 = 0; n0 < t.N; n0 += TN) tl.push_back(GemmTile{id, m0, n0});
    }
  }
  small_tasks.upload(sm, s);
  large_tasks.upload(lg, s);
  tiles.upload(tl, s);
  terms.upload(L.terms, s);
  n_small = int64_t(sm.size());
  n_large = int64_t(lg.size());
  n_tiles = int64_t(tl.size());
}

template <class T>
void run_gemm_tasks(const DevTaskList& L, const Bases<T>& b, int beta_zero, cudaStream_t s,
                    const int32_t* active) {
  if (L.n_small) {
    int64_t threads = L.n_small * kWarp;
    int blocks = int((threads + 255) / 256);
    k_gemm_small<T><<<blocks, 256, 0, s>>>(L.small_tasks.p, L.n_small, L.terms.p, b, beta_zero,
                                           active);
    DMRG_LAUNCHED();
  }
  if (L.n_tiles) {
    k_gemm_tiled<T><<<int(L.n_tiles), 256, 0, s>>>(L.tiles.p, L.large_tasks.p, L.terms.p, b,
                                                   beta_zero, active);
    DMRG_LAUNCHED();
  }
}
template void run_gemm_tasks<double>(const DevTaskList&, const Bases<double>&, int, cudaStream_t,
                                     const int32_t*);
template void run_gemm_tasks<float>(const DevTaskList&, const Bases<float>&, int, cudaStream_t,
                                    const int32_t*);

// ------------------------------------------------------------------------------------
// copy tasks (one warp per destination sub-block)
// ------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_copy(const CopyTask* __restrict__ tasks, int64_t n,
                                              const CopyTerm* __restrict__ terms, Bases<T> b) {
  int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / kWarp;
  int lane = threadIdx.x & (kWarp - 1);
  if (w >= n) return;
  const CopyTask t = tasks[w];
  T* D = b.p[t.dst.base] + t.dst.off;
  const int RC = t.rows * t.cols;
  for (int idx = lane; idx < RC; idx += kWarp) {
    int r = idx / t.cols, c = idx - r * t.cols;
    T acc = T(0);
    for (int j = t.t0; j < t.t1; ++j) {
      const CopyTerm g = terms[j];
      acc = fma(T(g.scale), b.p[g.src.base][g.src.off + (int64_t)r * g.src.ld + c], acc);
    }
    D[(int64_t)r * t.dst.ld + c] += acc;
  }
}

template <class T>
void run_copy_tasks(const CopyTask* d_tasks, int64_t n_tasks, const CopyTerm* d_terms,
                    const Bases<T>& b, cudaStream_t s) {
  if (!n_tasks) return;
  int blocks = int((n_tasks * kWarp + 255) / 256);
  k_copy<T><<<blocks, 256, 0, s>>>(d_tasks, n_tasks, d_terms, b);
  DMRG_LAUNCHED();
}
template void run_copy_tasks<double>(const CopyTask*, int64_t, const CopyTerm*,
                                     const Bases<double>&, cudaStream_t);
template void run_copy_tasks<float>(const CopyTask*, int64_t, const CopyTerm*,
                                    const Bases<float>&, cudaStream_t);

// ------------------------------------------------------------------------------------
// enlargement: one warp assembles one block of an enlarged operator from the block
// operators of the previous bond and the site operators of its W entries
// ------------------------------------------------------------------------------------
__constant__ int8_t c_op_entries[4][2][2] = {
    {{0, 0}, {1, 1}}, {{1, 1}, {-1, -1}}, {{1, 0}, {-1, -1}}, {{0, 1}, {-1, -1}}};

// One warp per enlarged block.  The block is made of up to four pieces (site states
// sigma_out, sigma_in), each the size of one source block; every contribution (W entry,
// site-operator element) fills one piece.  The lanes test 32 W entries at a time (source
// block lookup, Jordan-Wigner sign) and list the contributions per piece in shared memory,
// in entry order; each piece is then written once, its elements summed over its list in
// that order (the same sum, in the same order, as zero-filling and adding one by one).
constexpr int kEnlWarps = 8;
constexpr int kEnlCap = 64;   // contributions per piece and pass

__global__ void __launch_bounds__(kEnlWarps * 32) k_enlarge(const EnlBlock* __restrict__ blocks, int64_t n,
                                                 const int32_t* __restrict__ eptr,
                                                 const EntryDev* __restrict__ ents,
                                                 const int32_t* __restrict__ by_in, int nsrc,
                                                 const int64_t* __restrict__ boff,
                                                 const int32_t* __restrict__ dim,
                                                 const int32_t* __restrict__ npart,
                                                 const int8_t* __restrict__ lpar,
                                                 const LayDev* __restrict__ lay, int left,
                                                 const double* __restrict__ src,
                                                 double* __restrict__ out) {
  __shared__ int64_t s_off[kEnlWarps][4][kEnlCap];
  __shared__ double s_sc[kEnlWarps][4][kEnlCap];
  const int warp = threadIdx.x >> 5;
  const int64_t w = int64_t(blockIdx.x) * kEnlWarps + warp;
  const int lane = threadIdx.x & (kWarp - 1);
  if (w >= n) return;
  const EnlBlock b = blocks[w];
  const LayDev lo = lay[b.Qo], li = lay[b.Qi];
  double* dst = out + b.off;
  const int Di = li.D;
  const unsigned below = (1u << lane) - 1u;
  const int x_end = eptr[b.k + 1];
  int x0 = eptr[b.k];
  bool first = true;   // the first pass writes, later passes (long lists) add
  while (first || x0 < x_end) {
    int cnt[4] = {0, 0, 0, 0};
    while (x0 < x_end) {
      const int x = x0 + lane;
      int pc[2] = {-1, -1}, sbv[2] = {-1, -1};
      double scv[2] = {0.0, 0.0};
      if (x < x_end) {
        const EntryDev e = ents[x];
        for (int y = 0; y < 2; ++y) {
          const int so = c_op_entries[e.op][y][0], si = c_op_entries[e.op][y][1];
          if (so < 0) continue;
          const int qo = so ? lo.pblk1 : lo.pblk0, qi = si ? li.pblk1 : li.pblk0;
          if (qo < 0 || qi < 0) continue;
          const int sb = by_in[int64_t(e.src) * nsrc + qi];
          if (sb < 0) continue;
          double sc = e.coef;
          if (left) {
            if (e.op >= 2 && (npart[qi] & 1)) sc = -sc;
          } else {
            if (si && lpar[e.src]) sc = -sc;
          }
          pc[y] = 2 * so + si;
          sbv[y] = sb;
          scv[y] = sc;
        }
      }
      unsigned mask[4];
      bool fits = true;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        mask[p] = __ballot_sync(0xffffffffu, pc[0] == p || pc[1] == p);
        fits = fits && cnt[p] + __popc(mask[p]) <= kEnlCap;
      }
      if (!fits) break;   // this chunk opens the next pass
      for (int y = 0; y < 2; ++y) {
        if (pc[y] < 0) continue;
        const int p = pc[y];
        const int slot = cnt[p] + __popc(mask[p] & below);
        s_off[warp][p][slot] = boff[sbv[y]];
        s_sc[warp][p][slot] = scv[y];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) cnt[p] += __popc(mask[p]);
      x0 += kWarp;
    }
    __syncwarp();
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int so = p >> 1, si = p & 1;
      const int rows = so ? lo.D - lo.poff1 : lo.poff1;
      const int cols = si ? li.D - li.poff1 : li.poff1;
      if (rows <= 0 || cols <= 0 || (!first && cnt[p] == 0)) continue;
      const int ro = so ? lo.poff1 : 0, ri = si ? li.poff1 : 0;
      const int64_t* offs = s_off[warp][p];
      const double* scs = s_sc[warp][p];
      for (int idx = lane; idx < rows * cols; idx += kWarp) {
        const int r = idx / cols, cc = idx - r * cols;
        double* d = dst + (int64_t)(ro + r) * Di + ri + cc;
        double acc = first ? 0.0 : *d;
        for (int j = 0; j < cnt[p]; ++j) acc += scs[j] * src[offs[j] + idx];
        *d = acc;
      }
    }
    __syncwarp();
    first = false;
  }
}

void enlarge_blocks(const EnlBlock* blocks, int64_t n, const int32_t* eptr, const EntryDev* ents,
                    const int32_t* src_by_in, int src_nsec, const int64_t* src_boff,
                    const int32_t* src_dim, const int32_t* src_npart, const int8_t* src_lpar,
                    const LayDev* lay, int left, const double* src, double* out, cudaStream_t s) {
  if (n <= 0) return;
  k_enlarge<<<int((n + kEnlWarps - 1) / kEnlWarps), kEnlWarps * 32, 0, s>>>(blocks, n, eptr, ents, src_by_in, src_nsec,
                                                       src_boff, src_dim, src_npart, src_lpar, lay,
                                                       left, src, out);
  DMRG_LAUNCHED();
}

// x[pos[i]] = 1 (identity isometries)
__global__ void k_set_ones(double* __restrict__ x, const int64_t* __restrict__ pos, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[pos[i]] = 1.0;
}
void set_ones(double* x, const int64_t* pos, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  k_set_ones<<<int(std::min<int64_t>((n + 255) / 256, 1024)), 256, 0, s>>>(x, pos, n);
  DMRG_LAUNCHED();
}

// ------------------------------------------------------------------------------------
// vector kernels
// ------------------------------------------------------------------------------------
constexpr int kDotBlocks = 264;   // fixed grid => fixed reduction order
constexpr int kDotThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < int(blockDim.x >> 5); ++i) r += sh[i];
  return r;   // valid in thread 0
}

__global__ void k_multidot_partial(const double* const* vecs, int k, const double* __restrict__ w,
                                   int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  int64_t i0 = int64_t(blockIdx.x) * chunk, i1 = min(n, i0 + chunk);
  for (int j = 0; j < k; ++j) {
    const double* v = vecs[j];
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(v[i], w[i], s);
    double r = block_sum(s, sh);
    if (threadIdx.x == 0) part[j * gridDim.x + blockIdx.x] = r;
  }
}

__global__ void k_multidot_final(const double* __restrict__ part, int k, int nb,
                                 double* __restrict__ out) {
  int j = blockIdx.x;
  if (j >= k) return;
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[j * nb + i];
  double r = block_sum(s, sh);
  if (threadIdx.x == 0) out[j] = r;
}

void multidot(const double* const* d_vecs, int k, const double* w, int64_t n, double* d_out,
              double* d_partials, cudaStream_t s) {
  if (k <= 0) return;
  k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(d_vecs, k, w, n, d_partials);
  DMRG_LAUNCHED();
  k_multidot_final<<<k, 256, 0, s>>>(d_partials, k, kDotBlocks, d_out);
  DMRG_LAUNCHED();
}

__global__ void k_lincomb(const double* const* vecs, const double* __restrict__ coef, int k,
                          int64_t n, double* __restrict__ out, double beta, double cscale) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    double s = beta == 0.0 ? 0.0 : beta * out[i];
    for (int j = 0; j < k; ++j) s = fma(cscale * coef[j], vecs[j][i], s);
    out[i] = s;
  }
}

void lincomb(const double* const* d_vecs, const double* d_coef, int k, int64_t n, double* out,
             double beta_out, double coef_scale, cudaStream_t s) {
  int blocks = int(std::min<int64_t>((n + 255) / 256, 152 * 16));
  if (blocks < 1) blocks = 1;
  k_lincomb<<<blocks, 256, 0, s>>>(d_vecs, d_coef, k, n, out, beta_out, coef_scale);
  DMRG_LAUNCHED();
}

__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                              int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  int64_t i0 = int64_t(blockIdx.x) * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(a[i], b[i], s);
  double r = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}

void dot(const double* a, const double* b, int64_t n, double* d_out, double* d_partials,
         cudaStream_t s) {
  k_dot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, n, d_partials);
  DMRG_LAUNCHED();
  k_multidot_final<<<1, 256, 0, s>>>(d_partials, 1, kDotBlocks, d_out);
  DMRG_LAUNCHED();
}

__global__ void k_residual(const double* __restrict__ x, const double* __restrict__ Ax,
                           const double* __restrict__ theta, int64_t n, double* __restrict__ r) {
  double th = *theta;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    r[i] = Ax[i] - th * x[i];
}

void davidson_residual(const double* x, const double* Ax, const double* d_theta, int64_t n,
                       double* r, cudaStream_t s) {
  int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
  k_residual<<<blocks, 256, 0, s>>>(x, Ax, d_theta, n, r);
  DMRG_LAUNCHED();
}

__global__ void k_correction(const double* __restrict__ r, const double* __restrict__ diag,
                             const double* __restrict__ theta, int64_t n, double* __restrict__ t) {
  double th = *theta;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    double den = th - diag[i];
    if (fabs(den) < 1e-8) den = den < 0.0 ? -1e-8 : 1e-8;
    t[i] = r[i] / den;
  }
}

void davidson_correction(const double* r, const double* diag, const double* d_theta, int64_t n,
                         double* t, cudaStream_t s) {
  int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
  k_correction<<<blocks, 256, 0, s>>>(r, diag, d_theta, n, t);
  DMRG_LAUNCHED();
}

__global__ void k_scale(double* __restrict__ x, int64_t n, const double* __restrict__ sc,
                        int invert_sqrt) {
  double f = *sc;
  if (invert_sqrt) f = 1.0 / sqrt(f);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= f;
}

void scale_vec(double* x, int64_t n, const double* d_scale, int invert_sqrt, cudaStream_t s) {
  int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
  k_scale<<<blocks, 256, 0, s>>>(x, n, d_scale, invert_sqrt);
  DMRG_LAUNCHED();
}

__global__ void k_fill(double* __restrict__ x, int64_t n, double v) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] = v;
}

void fill_value(double* x, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return;
  int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)));
  k_fill<<<blocks, 256, 0, s>>>(x, n, v);
  DMRG_LAUNCHED();
}

// ------------------------------------------------------------------------------------
// diagonal of H_eff
// ------------------------------------------------------------------------------------
__global__ void k_heff_diag(const DiagTask* __restrict__ tasks, int n_tasks,
                            const DiagTerm* __restrict__ terms, const double* __restrict__ L,
                            const double* __restrict__ R, double* __restrict__ out) {
  int ti = blockIdx.x;
  if (ti >= n_tasks) return;
  const DiagTask t = tasks[ti];
  const int n = t.dL * t.dR;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    int l = idx / t.dR, r = idx - l * t.dR;
    double s = 0.0;
    for (int j = t.t0; j < t.t1; ++j) {
      const DiagTerm g = terms[j];
      s = fma(L[g.loff + (int64_t)l * (g.ldl + 1)], R[g.roff + (int64_t)r * (g.ldr + 1)], s);
    }
    out[t.psi_off + idx] = s;
  }
}

void heff_diag(const DiagTask* d_tasks, int n_tasks, const DiagTerm* d_terms,
               const double* lops, const double* rops, double* out, cudaStream_t s) {
  if (!n_tasks) return;
  k_heff_diag<<<n_tasks, 128, 0, s>>>(d_tasks, n_tasks, d_terms, lops, rops, out);
  DMRG_LAUNCHED();
}

// ------------------------------------------------------------------------------------
// symmetric eigensolver: parallel cyclic Jacobi (round-robin pairing), one block per matrix
// A (n x n, row-major, overwritten: diagonal -> eigenvalues), V (n x n) eigenvectors in
// columns.  Rotation of (Numerical Recipes): theta = (a_qq - a_pp) / (2 a_pq),
// t = sgn(theta)/(|theta| + sqrt(theta^2+1)), c = 1/sqrt(t^2+1), s = t c, A' = P^T A P.
// ------------------------------------------------------------------------------------
__device__ void jacobi_block(double* A, double* V, int n, double* cs, int* pp, int* qq,
                             double* red) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n * n; i += nt) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  if (n <= 1) return;
  const int m = (n + 1) & ~1;   // even number of players (a dummy when n is odd)
  for (int sweep = 0; sweep < 40; ++sweep) {
    // convergence: off-diagonal Frobenius norm against the full norm
    double off = 0.0, tot = 0.0;
    for (int i = tid; i < n * n; i += nt) {
      double a = A[i];
      tot += a * a;
      if (i / n != i % n) off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = off;
      red[2 * (tid >> 5) + 1] = tot;
    }
    __syncthreads();
    if (tid == 0) {
      double o2 = 0.0, t2 = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) { o2 += red[2 * w]; t2 += red[2 * w + 1]; }
      red[64] = (o2 <= 1e-30 * t2 || t2 == 0.0) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (red[64] != 0.0) break;
    for (int r = 0; r < m - 1; ++r) {
      // round-robin tournament: player m-1 fixed, the others rotate
      for (int k = tid; k < m / 2; k += nt) {
        int a, b;
        if (k == 0) {
          a = m - 1;
          b = r;
        } else {
          a = (r + k) % (m - 1);
          b = (r - k + (m - 1)) % (m - 1);
        }
        int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = A[p * n + q];
          if (apq != 0.0) {
            double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        pp[k] = p;
        qq[k] = q;
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
      }
      __syncthreads();
      // rows: A <- P^T A
      for (int e = tid; e < (m / 2) * n; e += nt) {
        int k = e / n, col = e - k * n;
        int p = pp[k], q = qq[k];
        if (q >= n) continue;
        double c = cs[2 * k], s = cs[2 * k + 1];
        if (s == 0.0) continue;
        double ap = A[p * n + col], aq = A[q * n + col];
        A[p * n + col] = c * ap - s * aq;
        A[q * n + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A P ; V <- V P
      for (int e = tid; e < (m / 2) * n; e += nt) {
        int k = e / n, row = e - k * n;
        int p = pp[k], q = qq[k];
        if (q >= n) continue;
        double c = cs[2 * k], s = cs[2 * k + 1];
        if (s == 0.0) continue;
        double ap = A[row * n + p], aq = A[row * n + q];
        A[row * n + p] = c * ap - s * aq;
        A[row * n + q] = s * ap + c * aq;
        double vp = V[row * n + p], vq = V[row * n + q];
        V[row * n + p] = c * vp - s * vq;
        V[row * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// rank-sort of eigenpairs (descending or ascending), ties by original index; clip <0 to 0
// when requested; eigenvector sign: largest |component| positive (lowest row on ties)
__device__ void sort_and_fix(const double* A, const double* V, int n, double* w_out,
                             double* V_out, int descending, int clip, int rs, int cs_) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double wi = A[i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double wj = A[j * n + j];
      bool before = descending ? (wj > wi) : (wj < wi);
      if (before || (wj == wi && j < i)) ++rank;
    }
    w_out[rank] = (clip && wi < 0.0) ? 0.0 : wi;
    // sign of column i
    int best = 0;
    double bv = -1.0;
    for (int rr = 0; rr < n; ++rr) {
      double a = fabs(V[rr * n + i]);
      if (a > bv) { bv = a; best = rr; }
    }
    double sg = V[best * n + i] < 0.0 ? -1.0 : 1.0;
    for (int rr = 0; rr < n; ++rr) V_out[rr * rs + rank * cs_] = sg * V[rr * n + i];
  }
}

// Matrices up to kEighSmem on a side are decomposed in shared memory (the rotations touch
// every element of two rows and two columns per round); larger ones in their global
// workspace.
constexpr int kEighSmem = 64;
constexpr size_t kEighSmemBytes = sizeof(double) * 2 * kEighSmem * kEighSmem;

// w offsets are provided separately to keep the kernel general
__global__ void __launch_bounds__(256) k_batched_eigh2(const int64_t* __restrict__ off,
                                                       const int64_t* __restrict__ woff,
                                                       const int32_t* __restrict__ dim,
                                                       double* A, double* V, double* Vs,
                                                       double* w, int descending, int clip) {
  extern __shared__ double eigh_sm[];
  __shared__ double cs[1024];
  __shared__ int pp[512], qq[512];
  __shared__ double red[80];
  int s = blockIdx.x;
  int n = dim[s];
  if (n <= 0) return;
  int64_t o = off[s];
  double* Aw = A + o;
  double* Vw = V + o;
  if (n <= kEighSmem) {
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) eigh_sm[i] = Aw[i];
    Aw = eigh_sm;
    Vw = eigh_sm + n * n;
    __syncthreads();
  }
  jacobi_block(Aw, Vw, n, cs, pp, qq, red);
  __syncthreads();
  sort_and_fix(Aw, Vw, n, w + woff[s], Vs + o, descending, clip, n, 1);
}

static void eigh_smem_attr() {
  static std::once_flag once;
  std::call_once(once, [] {
    DMRG_CUDA(cudaFuncSetAttribute(k_batched_eigh2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(kEighSmemBytes)));
  });
}

void batched_eigh2(const int64_t* d_off, const int64_t* d_woff, const int32_t* d_dim, int n,
                   double* d_A, double* d_V, double* d_Vs, double* d_w, int descending, int clip,
                   cudaStream_t s) {
  if (n <= 0) return;
  eigh_smem_attr();
  k_batched_eigh2<<<n, 256, kEighSmemBytes, s>>>(d_off, d_woff, d_dim, d_A, d_V, d_Vs, d_w,
                                                  descending, clip);
  DMRG_LAUNCHED();
}

// Ritz problem: H (k x k, leading dimension ld) -> ascending eigenvalues w, eigenvectors Y
// (k x k, column j = j-th lowest, sign fixed); k <= 64, decomposed in shared memory
__global__ void k_ritz(const double* __restrict__ H, int ld, int k, double* w, double* Y) {
  extern __shared__ double ritz_sm[];
  __shared__ double cs[1024];
  __shared__ int pp[512], qq[512];
  __shared__ double red[80];
  double* A = ritz_sm;
  double* V = ritz_sm + k * k;
  for (int i = threadIdx.x; i < k * k; i += blockDim.x) {
    int r = i / k, c = i - r * k;
    // symmetric from the lower triangle: row j holds <v_i, H v_j> for i <= j
    A[i] = (r >= c) ? H[r * ld + c] : H[c * ld + r];
  }
  __syncthreads();
  jacobi_block(A, V, k, cs, pp, qq, red);
  __syncthreads();
  // Y row j = coefficients of the j-th lowest Ritz vector (leading dimension 64)
  sort_and_fix(A, V, k, w, Y, 0, 0, 1, 64);
}

void ritz_solve(const double* d_H, int ld, int k, double* d_scratch, double* d_w, double* d_Y,
                cudaStream_t s) {
  (void)d_scratch;
  DMRG_REQUIRE(k >= 1 && k <= kEighSmem, DMRG_EINVAL, "internal: Ritz problem too large");
  static std::once_flag once;
  std::call_once(once, [] {
    DMRG_CUDA(cudaFuncSetAttribute(k_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(kEighSmemBytes)));
  });
  k_ritz<<<1, 256, sizeof(double) * 2 * k * k, s>>>(d_H, ld, k, d_w, d_Y);
  DMRG_LAUNCHED();
}

// ------------------------------------------------------------------------------------
// selection: k-th largest of w[0..n) by a descending bitonic sort in one block
// ------------------------------------------------------------------------------------
// bitonic sort (descending) of w padded to np2 with -inf, in shared memory when it fits
constexpr int64_t kKthSmem = 16384;

// out[0] = the k-th largest weight.  Fixed count (target <= 0): k = kmax.  Dynamic block
// state selection (target > 0): k = the smallest count in [kmin, kmax] whose discarded
// weight 1 - (w_1 + ... + w_k) (sorted descending, summed in that order in FP64) is at
// most target, else kmax.  out[1] = k.
__global__ void k_kth_largest(const double* __restrict__ w, int64_t n, int64_t kmax, int64_t kmin,
                              double target, double* gbuf, int64_t np2, double* out) {
  extern __shared__ double kth_sm[];
  double* buf = np2 <= kKthSmem ? kth_sm : gbuf;
  for (int64_t i = threadIdx.x; i < np2; i += blockDim.x) buf[i] = i < n ? w[i] : -INFINITY;
  __syncthreads();
  for (int64_t size = 2; size <= np2; size <<= 1) {
    for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (int64_t i = threadIdx.x; i < np2; i += blockDim.x) {
        int64_t j = i ^ stride;
        if (j > i) {
          bool desc = (i & size) == 0;
          double a = buf[i], b = buf[j];
          if (desc ? (a < b) : (a > b)) {
            buf[i] = b;
            buf[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    int64_t k = kmax;
    if (target > 0.0) {
      double kept = 0.0;
      for (int64_t i = 0; i < kmax; ++i) {
        kept += buf[i];
        if (i + 1 >= kmin && 1.0 - kept <= target) {
          k = i + 1;
          break;
        }
      }
    }
    out[0] = buf[k - 1];
    out[1] = double(k);
  }
}
void kth_largest(const double* w, int64_t n, int64_t kmax, int64_t kmin, double target,
                 double* d_scratch, double* out, cudaStream_t s) {
  DMRG_REQUIRE(kmax >= 1 && kmax <= n && kmin >= 1, DMRG_EINVAL, "internal: bad selection count");
  int64_t np2 = 1;
  while (np2 < n) np2 <<= 1;
  static std::once_flag once;
  std::call_once(once, [] {
    DMRG_CUDA(cudaFuncSetAttribute(k_kth_largest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(sizeof(double) * kKthSmem)));
  });
  const size_t smem = np2 <= kKthSmem ? sizeof(double) * size_t(np2) : 0;
  k_kth_largest<<<1, 1024, smem, s>>>(w, n, kmax, kmin, target, d_scratch, np2, out);
  DMRG_LAUNCHED();
}

// kept count and kept weight per sector: w sorted descending inside each sector
__global__ void k_count_kept(const int64_t* __restrict__ woff, const int32_t* __restrict__ dim,
                             int nsec, const double* __restrict__ w,
                             const double* __restrict__ lamM, int32_t* kept, double* kw) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsec) return;
  // keep every weight >= lambda_M (1 - 1e-10) (whole multiplets at the cut), never zeros
  double t = fmax(lamM[0] * (1.0 - 1e-10), 1e-14);
  int n = dim[s];
  const double* ws = w + woff[s];
  int c = 0;
  double sum = 0.0;
  while (c < n && ws[c] >= t) { sum += ws[c]; ++c; }
  kept[s] = c;
  kw[s] = sum;
}

void count_kept(const int64_t* d_woff, const int32_t* d_dim, int nsec, const double* w,
                const double* d_thr, int32_t* d_kept, double* d_kept_weight, cudaStream_t s) {
  if (nsec <= 0) return;
  k_count_kept<<<(nsec + 127) / 128, 128, 0, s>>>(d_woff, d_dim, nsec, w, d_thr, d_kept,
                                                  d_kept_weight);
  DMRG_LAUNCHED();
}

// U (D x m, row-major) = first m columns of the sorted, sign-fixed eigenvectors Vs (D x D)
__global__ void k_gather_u(const int64_t* __restrict__ voff, const int32_t* __restrict__ dim,
                           const int32_t* __restrict__ kept, const int64_t* __restrict__ uoff,
                           const double* __restrict__ Vs, double* __restrict__ U) {
  int s = blockIdx.x;
  int n = dim[s], m = kept[s];
  const double* v = Vs + voff[s];
  double* u = U + uoff[s];
  for (int i = threadIdx.x; i < n * m; i += blockDim.x) {
    int r = i / m, c = i - r * m;
    u[i] = v[r * n + c];
  }
}

void gather_u(const int64_t* d_voff, const int32_t* d_dim, const int32_t* d_kept,
              const int64_t* d_uoff, int nsec, const double* Vs, double* U, cudaStream_t s) {
  if (nsec <= 0) return;
  k_gather_u<<<nsec, 128, 0, s>>>(d_voff, d_dim, d_kept, d_uoff, Vs, U);
  DMRG_LAUNCHED();
}

// FP64 -> FP32 conversion (operator shadows of the mixed-precision path)
__global__ void k_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] = float(x[i]);
}
__global__ void k_to_f64(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    y[i] = double(x[i]);
}
void to_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)));
  k_to_f32<<<blocks, 256, 0, s>>>(x, y, n);
  DMRG_LAUNCHED();
}
void to_f64(const float* x, double* y, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  int blocks = int(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)));
  k_to_f64<<<blocks, 256, 0, s>>>(x, y, n);
  DMRG_LAUNCHED();
}

}  // namespace dmrg
