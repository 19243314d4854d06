// Internal definitions shared by the translation units of libdmrg (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <array>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/dmrg.h"

namespace dmrg {

extern std::atomic<int64_t> g_launches;
// host -> device uploads of bookkeeping tables (bytes, host nanoseconds blocked in the copy)
extern std::atomic<int64_t> g_upload_bytes, g_upload_ns;
// device allocations that missed the caching pool (count, host nanoseconds in cudaMalloc)
extern std::atomic<int64_t> g_malloc_count, g_malloc_ns;

// ---------------------------------------------------------------------------------------
// errors: every failure inside the library throws Error; the C-ABI turns it into a status
// ---------------------------------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define DMRG_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::dmrg::Error(DMRG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// every kernel launch of the library is followed by DMRG_LAUNCHED(): error check + count
#define DMRG_LAUNCHED()                                 \
  do {                                                  \
    DMRG_CUDA(cudaGetLastError());                      \
    ::dmrg::g_launches.fetch_add(1, std::memory_order_relaxed); \
  } while (0)

#define DMRG_REQUIRE(cond, code, msg)                 \
  do {                                                \
    if (!(cond)) throw ::dmrg::Error((code), (msg)); \
  } while (0)

// ---------------------------------------------------------------------------------------
// quantum numbers q = (N_p, N_n, 2M)
// ---------------------------------------------------------------------------------------
struct QN {
  int32_t a, b, m;
};
inline bool operator<(const QN& x, const QN& y) {
  if (x.a != y.a) return x.a < y.a;
  if (x.b != y.b) return x.b < y.b;
  return x.m < y.m;
}
inline bool operator==(const QN& x, const QN& y) { return x.a == y.a && x.b == y.b && x.m == y.m; }
inline bool operator!=(const QN& x, const QN& y) { return !(x == y); }
inline QN operator+(const QN& x, const QN& y) { return {x.a + y.a, x.b + y.b, x.m + y.m}; }
inline QN operator-(const QN& x, const QN& y) { return {x.a - y.a, x.b - y.b, x.m - y.m}; }
inline int particles(const QN& q) { return q.a + q.b; }

// sorted sector list with dimensions
struct SectorSet {
  std::vector<QN> q;
  std::vector<int> d;
  int find(const QN& x) const {
    auto it = std::lower_bound(q.begin(), q.end(), x);
    if (it == q.end() || *it != x) return -1;
    return int(it - q.begin());
  }
  int size() const { return int(q.size()); }
  int64_t total() const {
    int64_t t = 0;
    for (int x : d) t += x;
    return t;
  }
};

// ---------------------------------------------------------------------------------------
// device memory: a per-context caching pool.  All device work of a context runs on its one
// stream, so a block returned to the pool may be handed out again at once (stream order
// keeps the earlier users ahead).  Blocks are kept in power-of-two classes and released
// with cudaFree only when the context is destroyed (or a cudaMalloc fails).
// ---------------------------------------------------------------------------------------
struct Pool {
  std::vector<std::pair<size_t, void*>> free_blocks;   // (class bytes, pointer)
  size_t cached = 0;
  ~Pool() { trim(); }
  void trim() {
    for (auto& b : free_blocks) cudaFree(b.second);
    free_blocks.clear();
    cached = 0;
  }
  static size_t cls(size_t bytes) {
    size_t c = 256;
    while (c < bytes) c <<= 1;
    return c;
  }
  void* get(size_t bytes, size_t* got) {
    const size_t c = cls(bytes);
    for (size_t i = free_blocks.size(); i-- > 0;)
      if (free_blocks[i].first == c) {
        void* p = free_blocks[i].second;
        free_blocks[i] = free_blocks.back();
        free_blocks.pop_back();
        cached -= c;
        *got = c;
        return p;
      }
    void* p = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaMalloc(&p, c);
    g_malloc_ns.fetch_add(std::chrono::duration_cast<std::chrono::nanoseconds>(
                              std::chrono::steady_clock::now() - t0).count(),
                          std::memory_order_relaxed);
    g_malloc_count.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      trim();
      e = cudaMalloc(&p, c);
    }
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      throw Error(DMRG_ENOMEM, "cudaMalloc of " + std::to_string(c) + " bytes failed");
    }
    *got = c;
    return p;
  }
  void put(void* p, size_t c) {
    free_blocks.push_back({c, p});
    cached += c;
  }
};

// the pool of the context whose C-ABI call is running on this thread (nullptr: plain
// cudaMalloc / cudaFree)
extern thread_local Pool* tl_pool;

template <class T>
struct DevBuf {
  T* p = nullptr;
  int64_t n = 0;
  size_t cls = 0;
  Pool* pool = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), cls(o.cls), pool(o.pool) {
    o.p = nullptr;
    o.n = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      n = o.n;
      cls = o.cls;
      pool = o.pool;
      o.p = nullptr;
      o.n = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) {
      if (pool) pool->put(p, cls);
      else cudaFree(p);
    }
    p = nullptr;
    n = 0;
  }
  void alloc(int64_t count) {
    if (count <= n && p) return;
    release();
    if (count > 0) {
      const size_t bytes = sizeof(T) * size_t(count);
      pool = tl_pool;
      if (pool) {
        size_t got = 0;
        p = static_cast<T*>(pool->get(bytes, &got));
        cls = got;
        n = int64_t(got / sizeof(T));
      } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
          p = nullptr;
          (void)cudaGetLastError();
          throw Error(DMRG_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
        n = count;
      }
    }
  }
  void upload(const T* h, int64_t count, cudaStream_t s) {
    alloc(count);
    if (count) {
      const auto t0 = std::chrono::steady_clock::now();
      DMRG_CUDA(cudaMemcpyAsync(p, h, sizeof(T) * count, cudaMemcpyHostToDevice, s));
      g_upload_ns.fetch_add(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                std::chrono::steady_clock::now() - t0).count(),
                            std::memory_order_relaxed);
      g_upload_bytes.fetch_add(int64_t(sizeof(T)) * count, std::memory_order_relaxed);
    }
  }
  void upload(const std::vector<T>& h, cudaStream_t s) { upload(h.data(), int64_t(h.size()), s); }
};

// ---------------------------------------------------------------------------------------
// generic grouped GEMM task lists:  C (M x N) += sum_terms alpha op(A) op(B)
// operands are (base index, element offset, leading dimension) so that one list serves
// any set of base pointers (wave-function vectors change between Davidson products)
// ---------------------------------------------------------------------------------------
enum Base : int32_t {
  B_LOPS = 0,   // enlarged left operators
  B_ROPS = 1,   // enlarged right operators
  B_X = 2,      // input vector / matrix
  B_Y = 3,      // output
  B_T = 4,      // scratch
  B_U = 5,      // isometries
  B_V = 6,      // isometries (second set)
  B_Z = 7,      // extra
  NBASE = 8
};

struct Operand {
  int64_t off;
  int32_t base;
  int32_t ld;
};
struct GemmTerm {
  Operand A, B;
  int32_t K;
  int32_t trans;   // bit0: A transposed (A stored K x M), bit1: B transposed (B stored N x K)
  double alpha;
};
struct GemmTask {
  Operand C;
  int32_t M, N;
  int32_t t0, t1;   // terms [t0, t1)
};
// tile of a large task for the shared-memory kernel
struct GemmTile {
  int32_t task;
  int32_t m0, n0;
};

template <class T>
struct Bases {
  T* p[NBASE];
};

// host-side task list builder
struct TaskList {
  std::vector<GemmTask> tasks;
  std::vector<GemmTerm> terms;
  void begin_task(Operand C, int M, int N) {
    GemmTask t;
    t.C = C;
    t.M = M;
    t.N = N;
    t.t0 = int(terms.size());
    t.t1 = t.t0;
    tasks.push_back(t);
  }
  void add_term(Operand A, Operand B, int K, int trans, double alpha) {
    GemmTerm g;
    g.A = A;
    g.B = B;
    g.K = K;
    g.trans = trans;
    g.alpha = alpha;
    terms.push_back(g);
    tasks.back().t1 = int(terms.size());
  }
  void clear() { tasks.clear(); terms.clear(); }
};

// device-resident, split into small (warp per task) and large (tiled) parts
struct DevTaskList {
  DevBuf<GemmTask> small_tasks, large_tasks;
  DevBuf<GemmTerm> terms;
  DevBuf<GemmTile> tiles;
  int64_t n_small = 0, n_large = 0, n_tiles = 0;
  double flops = 0;      // algorithmic flops of the list
  // base_elems[b]: elements addressable through base b (0 = unused); every operand range
  // is checked against it on the host before the list reaches the device
  // small_limit: tasks of at most this many outputs run one warp each; the others are cut
  // into 64 x 64 tiles (0: every task tiled, the form the tensor-core engine wants)
  void build(const TaskList& L, const int64_t* base_elems, cudaStream_t s,
             int64_t small_limit = 1024);
};


// copy-scale tasks: dst (rows x cols, ld_dst) += sum_terms scale * src (rows x cols, ld_src)
struct CopyTerm {
  Operand src;
  double scale;
};
struct CopyTask {
  Operand dst;
  int32_t rows, cols;
  int32_t t0, t1;
};
struct CopyList {
  std::vector<CopyTask> tasks;
  std::vector<CopyTerm> terms;
};
void validate_copy_tasks(const CopyList& L, const int64_t* base_elems);

// ---------------------------------------------------------------------------------------
// kernels (kernels.cu)
// ---------------------------------------------------------------------------------------
// active (optional, device): the launch does nothing while active[0] == 0 (batch mode)
template <class T>
void run_gemm_tasks(const DevTaskList& L, const Bases<T>& b, int beta_zero, cudaStream_t s,
                    const int32_t* active = nullptr);
// the same task lists on the tensor cores (tgemm.cu): operands of types TA, TB (float or
// double) split into TF32 high + low parts, three MMAs per product, FP32 accumulation, C of
// type TC; tasks of at most 1024 outputs with FP32 FMAs on the CUDA cores
template <class TA, class TB, class TC>
void run_gemm_tasks_tc(const DevTaskList& L, const Bases<void>& b, int beta_zero, cudaStream_t s,
                       const int32_t* active = nullptr);
template <class T>
void run_copy_tasks(const CopyTask* d_tasks, int64_t n_tasks, const CopyTerm* d_terms,
                    const Bases<T>& b, cudaStream_t s);

// Davidson / vector kernels
void multidot(const double* const* d_vecs, int k, const double* w, int64_t n, double* d_out,
              double* d_partials, cudaStream_t s);
// out = beta out + coef_scale sum_j coef[j] vecs[j]
void lincomb(const double* const* d_vecs, const double* d_coef, int k, int64_t n, double* out,
             double beta_out, double coef_scale, cudaStream_t s);
// d_out[0] = a . b (fixed reduction order)
void dot(const double* a, const double* b, int64_t n, double* d_out, double* d_partials,
         cudaStream_t s);
void davidson_residual(const double* x, const double* Ax, const double* d_theta, int64_t n,
                       double* r, cudaStream_t s);
void davidson_correction(const double* r, const double* diag, const double* d_theta, int64_t n,
                         double* t, cudaStream_t s);
void scale_vec(double* x, int64_t n, const double* d_scale, int invert_sqrt, cudaStream_t s);
void fill_value(double* x, int64_t n, double v, cudaStream_t s);

// diagonal of H_eff: for each psi element the sum over diagonal-preserving terms
struct DiagTask {
  int64_t psi_off;
  int32_t dL, dR;
  int32_t t0, t1;
};
struct DiagTerm {
  int64_t loff, roff;   // diagonal blocks in the enlarged left / right operator arenas
  int32_t ldl, ldr;
};
void heff_diag(const DiagTask* d_tasks, int n_tasks, const DiagTerm* d_terms,
               const double* lops, const double* rops, double* out, cudaStream_t s);

// batched symmetric eigensolver (parallel cyclic Jacobi, FP64), one block per matrix:
// A at off[s] (n x n, destroyed), V scratch (n x n), Vs sorted sign-fixed eigenvectors,
// w at woff[s] (eigenvalues, descending or ascending, optionally clipped at 0)
void batched_eigh2(const int64_t* d_off, const int64_t* d_woff, const int32_t* d_dim, int n,
                   double* d_A, double* d_V, double* d_Vs, double* d_w, int descending, int clip,
                   cudaStream_t s);
void ritz_solve(const double* d_H, int ld, int k, double* d_scratch, double* d_w, double* d_Y,
                cudaStream_t s);
// eigenpairs of rho_Q = B B^T from the singular vectors of the wave-function block B
// (svd.cu): B = psi block (d x e, trans 0) or its transpose (trans 1, the block is e x d),
// [psi0 psi1] / sqrt(2) with two roots; eigenvalues descending at w_off, eigenvectors as
// the columns of a d x d row-major matrix at vs_off (largest |component| positive)
struct SvdJob {
  int64_t src;      // offset of the block in psi0 (and psi1)
  int64_t vs_off;   // output eigenvectors
  int64_t w_off;    // output eigenvalues
  int32_t D;        // sector dimension d
  int32_t e;        // the block's other dimension
  int32_t trans;
  int32_t roots;
};
size_t svd_smem_bytes(const SvdJob& j, int cluster);
size_t svd_smem_limit();   // largest dynamic shared memory of one CTA of the SVD kernel
// one cluster of `cluster` CTAs (1, 8 or 16) per job; *d_noconv = 1 if a job reached its
// sweep limit
void svd_jacobi(const SvdJob* d_jobs, int n_jobs, int cluster, size_t smem, const double* psi0,
                const double* psi1, double* w, double* vs, int* d_noconv, cudaStream_t s);
// a piece of a wave-function block paired with another (or itself): the sum over
// i < nr, j < nc of psi[a + i lda + j] psi[b + i ldb + j] goes to sum number slot (0..4)
struct RdmTask {
  int64_t a, b;
  int32_t lda, ldb, nr, nc, slot, pad;
};
// the five sums of the dot density matrix; d_part holds one double per task
void rdm_sums(const RdmTask* d_tasks, int64_t n, const double* psi, double* d_part,
              double* d_out, cudaStream_t s);

// all-pairs mutual information (mutual.cu): rectangle dot products (lda < 0: trace of the
// B rectangle), their sums per slot (slots = consecutive task ranges), and the embedding of
// operator blocks (src < 0: an identity) into the blocks of an enlarged operator
struct RectDot {
  int64_t a, b;
  int32_t lda, ldb, nr, nc;
  double sign;
};
struct EmbedTask {
  int64_t src, dst;
  int32_t lds, ldd, nr, nc;
  double sign;
};
void rect_dots(const RectDot* d_tasks, int64_t n, const double* A, const double* B,
               double* d_part, cudaStream_t s);
void slot_sums(const int64_t* d_ptr, int64_t n_slots, const double* d_part, double* d_out,
               cudaStream_t s);
void embed_blocks(const EmbedTask* d_tasks, int64_t n, const double* S, double* D,
                  cudaStream_t s);
// global selection: k-th largest of w[0..n) (ties irrelevant for the value) in out[0] and k
// in out[1]; k = kmax, or with target > 0 the smallest k in [kmin, kmax] whose discarded
// weight 1 - (sum of the k largest) is at most target (kmax if none)
void kth_largest(const double* w, int64_t n, int64_t kmax, int64_t kmin, double target,
                 double* d_scratch, double* out, cudaStream_t s);
// kept[s] = number of w >= max(lambda_M (1 - 1e-10), 1e-14) in sector s (w descending)
void count_kept(const int64_t* d_woff, const int32_t* d_dim, int nsec, const double* w,
                const double* d_lamM, int32_t* d_kept, double* d_kept_weight, cudaStream_t s);
void gather_u(const int64_t* d_voff, const int32_t* d_dim, const int32_t* d_kept,
              const int64_t* d_uoff, int nsec, const double* Vs, double* U, cudaStream_t s);
void to_f32(const double* x, float* y, int64_t n, cudaStream_t s);
void to_f64(const float* x, double* y, int64_t n, cudaStream_t s);

// fused H_eff product (heff.cu): one term of an output block ...
struct HeffItem {
  int64_t loff, roff, xoff;   // L block (dLo x dLi), R block (dRo x dRi), psi_in block (dLi x dRi)
  int32_t dLi, dRi;
  float sign;                 // (-1)^{|R_k| N(Q_L)}
  int32_t pad;
};
// ... one unit of work: a group of terms of one output tile (rows r0..r0+m, columns
// c0..c0+n of the psi' block at yoff); written to psi' directly (poff < 0) or as a partial
// tile at poff of the scratch, summed later in group order
struct HeffTile {
  int64_t yoff;
  int64_t poff;
  int32_t ld;                 // dRo of the output block
  int32_t r0, c0, m, n;
  int32_t i0, i1;             // items [i0, i1)
  int32_t inst;               // instance (batch mode), 0 for one context
};
// deterministic sum of the partial tiles of one output tile
struct HeffRed {
  int64_t yoff, poff;
  int32_t ld, r0, c0, m, n, groups;
  int32_t inst, pad;
};
// base pointers of every instance of a fused launch (passed by value); active[inst] == 0
// makes the thread blocks of that instance return at once (batch mode)
constexpr int kMaxInst = 64;
template <class T>
struct HeffPtrs {
  const T* L[kMaxInst];
  const T* R[kMaxInst];
  const T* X[kMaxInst];
  T* Y[kMaxInst];
  T* P[kMaxInst];
  const int32_t* active;
};
// output blocks with m, n <= kSmallEdge whose terms all have dLi, dRi <= kSmallEdge go
// to the warp-per-tile CUDA-core product (heff_small.cu); its tiles are whole blocks
constexpr int kSmallEdge = 16;
// output blocks with a dimension of their own or of one of their terms above kBigEdge go to
// the grouped GEMM passes (tgemm.cu / kernels.cu) instead of the fused tile kernels
constexpr int kBigEdge = 128;
template <class T>
void heff_small(const HeffTile* d_tiles, int64_t n_tiles, const HeffItem* d_items,
                const HeffPtrs<T>& ptrs, cudaStream_t s);
template <class T>
void heff_reduce(const HeffRed* d_red, int64_t n_red, const HeffPtrs<T>& ptrs, cudaStream_t s);
// mixed path: the same product with 3xTF32 warp MMAs (heff_tc.cu)
void heff_tc(const HeffTile* d_tiles, int64_t n_tiles, const HeffItem* d_items,
             const HeffRed* d_red, int64_t n_red, const HeffPtrs<float>& ptrs, cudaStream_t s);
template <class TO>
void pad_psi(const double* x, TO* xp, const int64_t* src_off, const int64_t* dst_off,
             const int32_t* len, int nblocks, cudaStream_t s);
template <class T>
void heff_fused(const HeffTile* d_tiles, int64_t n_tiles, const HeffItem* d_items,
                const HeffRed* d_red, int64_t n_red, const HeffPtrs<T>& ptrs, cudaStream_t s);
// psi into / out of the 16-byte aligned staging copies, with the vector pointers read from
// device memory (*xp_ptr, *out_ptr) so that a captured graph can be replayed on new vectors
template <class TO>
void pad_psi_ind(const double* const* x_ptr, TO* xp, const int64_t* src_off,
                 const int64_t* dst_off, const int32_t* len, int nblocks, const int32_t* active,
                 cudaStream_t s);
template <class TI>
void out_to_f64_ind(const TI* y, double* const* out_ptr, int64_t n, const int32_t* active,
                    cudaStream_t s);

// enlargement of block operators by one site (kernels.cu)
struct EntryDev {
  int32_t src;     // source label
  int32_t op;      // site operator: 0 = 1, 1 = n, 2 = c+, 3 = c
  double coef;
};
struct EnlBlock {
  int64_t off;     // destination block offset
  int32_t k, Qo, Qi, pad;
};
struct LayDev {
  int32_t pblk0, pblk1, poff1, D;
};
// one operator block to renormalize: O (enlarged sectors so, si) at xoff -> O' at yoff,
// intermediate O U_i at toff of the scratch
struct ProjTask {
  int64_t xoff, yoff, toff;
  int32_t so, si;
};
// tile_beg1/2: [n + 1] prefix sums of the 32 x 32 tiles of stage 1 (D_o x m_i) and
// stage 2 (m_o x m_i) per block
void project_blocks(const ProjTask* tasks, const int64_t* tile_beg1, int64_t n_tiles1,
                    const int64_t* tile_beg2, int64_t n_tiles2, int64_t n, const int32_t* D,
                    const int32_t* m, const int64_t* uoff, const double* X, const double* U,
                    double* T, double* Y, cudaStream_t s);
// blocks with D_o, D_i <= 32 (one warp each, both products fused)
void set_ones(double* x, const int64_t* pos, int64_t n, cudaStream_t s);
void project_small(const ProjTask* tasks, int64_t n, const int32_t* D, const int32_t* m,
                   const int64_t* uoff, const double* X, const double* U, double* Y,
                   cudaStream_t s);
void enlarge_blocks(const EnlBlock* blocks, int64_t n, const int32_t* eptr, const EntryDev* ents,
                    const int32_t* src_by_in, int src_nsec, const int64_t* src_boff,
                    const int32_t* src_dim, const int32_t* src_npart, const int8_t* src_lpar,
                    const LayDev* lay, int left, const double* src, double* out, cudaStream_t s);

// learned preconditioner (mlp.cu)
template <class T>
struct MlpActs {
  DevBuf<T> Z1, H1, Z2, H2, Z3, H3, Y, dY, dH, dZ;
  DevBuf<double> part;
  int64_t cap = 0;
  void ensure(int64_t B) {
    if (B <= cap) return;
    const int64_t nh = B * 256;
    Z1.alloc(nh);
    H1.alloc(nh);
    Z2.alloc(nh);
    H2.alloc(nh);
    Z3.alloc(nh);
    H3.alloc(nh);
    dH.alloc(nh);
    dZ.alloc(nh);
    Y.alloc(B);
    dY.alloc(B);
    cap = B;
  }
};
int64_t mlp_n_params();
template <class T>
void mlp_forward(const T* P, const T* X, int64_t B, MlpActs<T>& a, cudaStream_t s);
template <class T>
double mlp_backward(const T* P, const T* X, const T* Tg, int64_t B, MlpActs<T>& a, T* G,
                    cudaStream_t s);
template <class T>
void mlp_adam(T* P, const T* G, T* m, T* v, int64_t n, double lr, int step, cudaStream_t s);
template <class T>
void mlp_gather(const T* S, const int32_t* idx, int64_t B, T* X, T* Tg, cudaStream_t s);
template <class T>
void mlp_features(const double* r, const double* x, const double* diag, const double* sc,
                  int64_t n, T* X, cudaStream_t s);
template <class T>
void mlp_output_to_double(const T* y, double* out, int64_t n, cudaStream_t s);
void mlp_harvest(const double* r, const double* x, const double* psi, const double* diag,
                 const double* sc, int64_t n, int64_t start, int64_t stride, int64_t count,
                 float* out, cudaStream_t s);
void mlp_err_vec(const double* x, const double* psi, const double* sc, int64_t n, double* e,
                 cudaStream_t s);

// read-only view of the H_eff task lists of the superblock currently set up at position p
// (nothing is built or allocated; false if the superblock at p is not set up)
// elements of the allocation-free product's file-scope intermediate (noalloc.cu): 2^21
// doubles = 16 MiB; the two-stage lists it needs are built only for superblocks that fit
constexpr int64_t kScratchElems = int64_t(1) << 21;
struct HeffView {
  const DevTaskList* st1;
  const DevTaskList* st2;
  const double* L;
  const double* R;
  int64_t size;
  int64_t t_elems;
  cudaStream_t stream;
  int device;               // the device the context was created on
  bool lists_ready;         // the two-stage lists exist (only when t_elems <= kScratchElems)
};
bool heff_view(dmrg_ctx* c, int p, HeffView* v);
void set_error(dmrg_ctx* c, const char* msg);

}  // namespace dmrg
