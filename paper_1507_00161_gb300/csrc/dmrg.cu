// libdmrg: two-site DMRG on the GPU for the shell-model Hamiltonian of Eq. (1).
//
// Host code here does the integer bookkeeping (sectors, block lists, term and tile
// tables); every floating-point step runs in kernels:
//   enlargement of block operators by one site (k_enlarge, kernels.cu), H_eff psi (fused
//   tile kernels: heff.cu FP64, heff_tc.cu split-TF32 tensor cores), Davidson vector
//   algebra and the Ritz problem, reduced density matrices, their eigendecomposition and
//   the selection of the kept states (kernels.cu), renormalization of every normal and
//   complementary operator (renorm.cu), and the prediction of the next wave function.
#include <malloc.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <exception>
#include <functional>
#include <initializer_list>
#include <memory>
#include <mutex>
#include <set>
#include <thread>

#include "common.h"
#include "problem.h"

namespace dmrg {

// ---------------------------------------------------------------------------------------
// block-sparse operator sets and enlarged layouts
// ---------------------------------------------------------------------------------------
struct OpBlock {
  int32_t so, si;
  int64_t off;
};

struct OpSet {
  SectorSet sec;
  int nlab = 0;
  std::vector<int64_t> lab_ptr;   // [nlab + 1]
  std::vector<OpBlock> blocks;
  DevBuf<double> data;
  DevBuf<float> data32;
  int64_t n_elems = 0;
  std::vector<int32_t> by_in;     // nlab x nsec: block index by input sector (or -1)
  // device copies used when this set is the source of an enlargement
  DevBuf<int32_t> d_by_in, d_dim, d_npart;
  DevBuf<int64_t> d_boff;
  bool dev_index_ready = false;
  void index_by_in() {
    dev_index_ready = false;
    by_in.assign(size_t(nlab) * sec.size(), -1);
    for (int k = 0; k < nlab; ++k)
      for (int64_t x = lab_ptr[k]; x < lab_ptr[k + 1]; ++x)
        by_in[size_t(k) * sec.size() + blocks[x].si] = int32_t(x);
  }
};

// enlarged space: block (x) site (left) or site (x) block (right); piece sigma = 0 first
struct Layout {
  SectorSet sec;
  std::vector<std::array<int, 2>> pblk;   // block sector of piece sigma (or -1)
  std::vector<std::array<int, 2>> poff;   // row offset of piece sigma
};

// O(1) sector lookup over the bounding box of a sector list
struct QIndex {
  int a0 = 0, b0 = 0, m0 = 0, na = 0, nb = 0, nm = 0;
  std::vector<int32_t> idx;
  explicit QIndex(const SectorSet& s) {
    if (s.q.empty()) return;
    int a1 = s.q[0].a, b1 = s.q[0].b, m1 = s.q[0].m;
    a0 = a1, b0 = b1, m0 = m1;
    for (auto& q : s.q) {
      a0 = std::min(a0, q.a), a1 = std::max(a1, q.a);
      b0 = std::min(b0, q.b), b1 = std::max(b1, q.b);
      m0 = std::min(m0, q.m), m1 = std::max(m1, q.m);
    }
    na = a1 - a0 + 1, nb = b1 - b0 + 1, nm = m1 - m0 + 1;
    idx.assign(size_t(na) * nb * nm, -1);
    for (int i = 0; i < s.size(); ++i)
      idx[(size_t(s.q[i].a - a0) * nb + (s.q[i].b - b0)) * nm + (s.q[i].m - m0)] = i;
  }
  int find(const QN& q) const {
    const int a = q.a - a0, b = q.b - b0, m = q.m - m0;
    if (a < 0 || a >= na || b < 0 || b >= nb || m < 0 || m >= nm) return -1;
    return idx[(size_t(a) * nb + b) * nm + m];
  }
};

// constant W entries of one site grouped by destination label
struct SiteEntries {
  std::vector<int32_t> ptr;
  std::vector<EntryDev> e;
  DevBuf<int32_t> dptr;
  DevBuf<EntryDev> de;
  bool ready = false;
};

// basis of a stored block: kept columns of an isometry per enlarged sector
struct Iso {
  Layout lay;
  std::vector<int> m;            // kept states per enlarged sector
  std::vector<int64_t> uoff;     // offset of U (D x m, row-major) per enlarged sector
  std::vector<int> kept_idx;     // enlarged sector -> stored sector index (or -1)
  std::vector<int> enl_idx;      // stored sector -> enlarged sector
  DevBuf<double> data;
  bool identity = false;         // every state kept unrotated (no truncation)
};

struct Blk {
  OpSet ops;
  Iso iso;
  bool valid = false;
  uint64_t gen = 0;   // changes whenever ops change (identifies the block for prefetching)
};

// host part of an enlargement: layout, destination block table, device tables to upload
struct EnlPlan {
  Layout lay;
  OpSet out;                                   // host tables only, no data
  std::vector<std::vector<EnlBlock>> part;     // destination blocks in label order
  std::vector<int64_t> pbase;
  std::vector<LayDev> ld;
  double det[8] = {};                          // host seconds of its phases
};

// enlargement planned ahead on a host thread while the GPU works on the previous step
struct Prefetch {
  std::thread th;
  bool active = false;
  int s = -1;
  bool left = false;
  uint64_t gen = 0;
  EnlPlan plan;
  std::exception_ptr err;
  // device part issued ahead on a stream of its own (dev_ready: out and lay hold the result,
  // complete once `done` has fired; the small tables live until then)
  bool dev_ready = false;
  Layout lay;
  OpSet out;
  DevBuf<LayDev> t_lay;
  DevBuf<EnlBlock> t_blocks;
  DevBuf<int8_t> t_par;
  cudaStream_t st = nullptr;
  cudaEvent_t ready = nullptr, done = nullptr;
};

struct Super {
  int p = -1;
  Layout Ll, Rl;
  OpSet L, R;
  std::vector<int> bL, bR, bdl, bdr;   // psi blocks: sector indices and dims
  std::vector<int64_t> boff;
  std::vector<int> psi_of_L, psi_of_R;
  int64_t size = 0;
  DevTaskList st1, st2;
  bool two_stage_ready = false;
  // output blocks too wide for the fused tile kernels (a dimension of the block or of one
  // of its terms above 32): two grouped GEMM passes, T_k = psi(b_in) R_k^T into a scratch,
  // then psi'(b_out) = sum_k s_k L_k T_k (every such output block written by one task)
  DevTaskList big1, big2;
  DevBuf<HeffRed> big_red;            // partial blocks of stage-2 term groups, added in order
  int64_t big_t_elems = 0, big_p_elems = 0, n_big_red = 0;
  int64_t n_big_blocks = 0;
  struct Term {
    int64_t lb, rb;
    int bin, bout;
    double sign;
  };
  std::vector<Term> terms_host;
  DevBuf<HeffItem> fitems;
  DevBuf<HeffTile> ftiles, stiles;   // tile kernels (32 x 32 tiles); small-block kernel
  DevBuf<HeffRed> fred;
  int64_t n_ftiles = 0, n_stiles = 0, n_fred = 0, p_elems = 0;
  std::vector<HeffItem> h_items;
  std::vector<HeffTile> h_tiles, h_stiles;
  std::vector<HeffRed> h_red;
  std::vector<double> h_cost, h_scost;
  // 16-byte aligned copy of psi used by the fused product
  std::vector<int64_t> pad_off;
  int64_t pad_size = 0;
  DevBuf<int64_t> d_src_off, d_pad_off;
  DevBuf<int32_t> d_pad_len;
  int64_t t_elems = 0;
  double flops = 0, bytes = 0;
  int64_t n_items = 0;
  DevBuf<DiagTask> dtasks;
  DevBuf<DiagTerm> dterms;
  int n_dtasks = 0;
  DevBuf<double> diag;
  bool diag_ready = false;
  // the product's kernels after the staging of psi, captured as a CUDA graph at the second
  // product of a precision (0 = FP64, 1 = mixed) on this superblock and replayed after that
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int64_t n_launches = 0;       // kernel nodes
    int64_t eager = 0, replays = 0;
    bool empty = false;           // the product launches no kernel here
    const void* key[6] = {};      // scratch pointers at capture
  } graph[2];
  Super() = default;
  Super(const Super&) = delete;
  Super& operator=(const Super&) = delete;
  ~Super() {
    // an executable graph still in flight is released when it completes
    for (auto& g : graph)
      if (g.exec) cudaGraphExecDestroy(g.exec);
  }
};

}  // namespace dmrg

struct dmrg_ctx {
  dmrg::Pool pool;   // first member: destroyed last, after every buffer returned to it
  std::string err = "no error";
  // wall seconds spent in the phases of a step (host bookkeeping + device work)
  double t_enlarge = 0, t_super = 0, t_davidson = 0, t_truncate = 0, t_project = 0,
         t_predict = 0;
  double t_sync = 0, t_enlarge_host = 0;   // host blocked on the stream; enlarge host walk
  int64_t last_sizes[5] = {0, 0, 0, 0, 0};   // last superblock: L, R blocks, terms, tiles, small tiles
  int64_t term_hist[8] = {};
  double kernel_flops = 0;     // last superblock: flops in the order the tile kernels use   // last superblock: terms by largest inner dim; flops share
  double t_detail[24] = {};   // finer host phases (see dmrg.h)
  dmrg::Chain chain;
  dmrg::MPO mpo;
  dmrg_options opt{};
  int dbss_min = 0;          // dynamic block state selection: M_min (0 = fixed M)
  double dbss_target = 0.0;  // and the discarded-weight target
  cudaStream_t stream = nullptr;
  int N = 0;
  int device = -1;             // the device current when the context was created
  std::vector<std::set<std::tuple<int, int, int>>> reach_left, reach_right;
  std::vector<dmrg::Blk> left, right;
  bool built = false;
  std::unique_ptr<dmrg::Super> sb;
  dmrg::Prefetch pf;
  // Davidson workspace
  dmrg::DevBuf<double> V, AV, r, t, x, Ax, x1, Ax1, r1, small, partials;
  dmrg::DevBuf<const double*> vptr;
  int64_t ws_n = 0, ws_sub = 0;
  // current eigenvector and what the next guess needs
  dmrg::DevBuf<double> psi, psi_guess;
  bool psi_valid = false;
  int psi_p = -1;
  // two-state targeting: the second state of the last step and its predicted guess
  int n_roots = 1;
  dmrg::DevBuf<double> psi1, psi_guess1;
  bool psi1_valid = false;
  std::unique_ptr<dmrg::Super> prev;   // layouts of the superblock psi belongs to
  // scratch
  dmrg::DevBuf<double> T, tmp, rho, eV, eVs, ew, sel;
  dmrg::DevBuf<int> noconv;    // set by a truncation SVD that reached its sweep limit
  int big_edge = dmrg::kBigEdge;   // output blocks wider than this: grouped GEMM passes (0: never)
  int svd_cluster = 0;         // forced cluster size of the truncation SVDs (0: per sector)
  int64_t eig_noconv = 0;      // truncations with such an SVD
  dmrg::DevBuf<float> f32a, f32b, f32T, part32;
  dmrg::DevBuf<double> part64, xpad64, ybat64, bigpart64, ygraph64;
  int heff_graph = 1;          // replay the product as a CUDA graph (0: eager launches)
  int64_t graph_replays = 0;   // products replayed from a graph
  cudaStream_t cap_stream = nullptr;   // graph capture
  dmrg::DevBuf<float> bigpart32;  // partial blocks of the stage-2 term groups
  dmrg::DevBuf<float> xpad32;
  // precomputed per-site W entry orders (grouped by destination label)
  std::vector<std::vector<int>> w_by_b, w_by_a;
  std::vector<dmrg::SiteEntries> ent_left, ent_right;
  std::vector<int32_t> order;   // chain position -> site of the problem
  // learned preconditioner: parameters, Adam moments, harvested samples, Davidson history
  dmrg::DevBuf<float> mlp_p, mlp_g, mlp_m, mlp_v, mlp_samples, mlp_X, mlp_T, mlp_feat;
  dmrg::MlpActs<float> mlp_acts;
  dmrg::DevBuf<int32_t> mlp_idx;
  bool mlp_ready = false, mlp_trained = false;
  int mlp_step = 0;
  int64_t mlp_nsamp = 0, mlp_cap = 262144, mlp_head = 0, mlp_calls = 0;
  int mlp_harvest = 0, mlp_per_iter = 2048;
  dmrg::DevBuf<double> hist_x, hist_r, hist_theta, hist_tmp, mlp_sc;
  // H_eff timing: event pairs recorded around every product, resolved after a sync
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  int64_t heff_products = 0;
  double heff_seconds = 0, heff_flops = 0, heff_bytes = 0;
  double step_heff_seconds = 0;
  // pinned host words for the small per-iteration readbacks (a copy into pageable memory
  // goes through a staging buffer of the driver)
  double* h_words = nullptr;
  // the FP64 Rayleigh quotient of the mixed path runs on a stream of its own, overlapping
  // the truncation that follows it (which does not need the energy)
  cudaStream_t rq_stream = nullptr;
  cudaEvent_t rq_in = nullptr, rq_out = nullptr;
  dmrg::DevBuf<double> rq_part;
  bool rq_pending = false, rq_todo = false;
  double* rq_target = nullptr;   // where a deferred energy goes (sweeps)
  dmrg::Super* rq_sb = nullptr;
  int64_t rq_n = 0;
  double* rq_sc = nullptr;
  ~dmrg_ctx() {
    if (pf.th.joinable()) pf.th.join();
    if (pf.st) {
      cudaStreamSynchronize(pf.st);
      cudaStreamDestroy(pf.st);
    }
    if (pf.ready) cudaEventDestroy(pf.ready);
    if (pf.done) cudaEventDestroy(pf.done);
    if (rq_stream) {
      cudaStreamSynchronize(rq_stream);
      cudaStreamDestroy(rq_stream);
    }
    if (rq_in) cudaEventDestroy(rq_in);
    if (rq_out) cudaEventDestroy(rq_out);
    for (auto e : ev) cudaEventDestroy(e);
    if (h_words) cudaFreeHost(h_words);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }
};

namespace dmrg {

thread_local Pool* tl_pool = nullptr;

static std::atomic<uint64_t> g_blk_gen{0};   // generations of stored blocks

using Ctx = dmrg_ctx;

static double wall() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
struct PhaseTimer {
  double& acc;
  double t0;
  explicit PhaseTimer(double& a) : acc(a), t0(wall()) {}
  ~PhaseTimer() { acc += wall() - t0; }
};

// host waits for the context stream (time accumulated in t_sync)
static void sync(Ctx& c) {
  const double t0 = wall();
  DMRG_CUDA(cudaStreamSynchronize(c.stream));
  c.t_sync += wall() - t0;
}

static bool reachable(const std::set<std::tuple<int, int, int>>& s, const QN& q) {
  return s.count(std::make_tuple(q.a, q.b, q.m)) > 0;
}

static void build_reach(Ctx& c) {
  const int N = c.N;
  c.reach_left.assign(N + 1, {});
  c.reach_right.assign(N + 1, {});
  c.reach_left[0].insert({0, 0, 0});
  for (int x = 0; x < N; ++x) {
    auto s = c.reach_left[x];
    for (auto& t : c.reach_left[x]) {
      QN q{std::get<0>(t), std::get<1>(t), std::get<2>(t)};
      QN r = q + c.chain.q[x];
      s.insert({r.a, r.b, r.m});
    }
    c.reach_left[x + 1] = s;
  }
  c.reach_right[N].insert({0, 0, 0});
  for (int x = N - 1; x >= 0; --x) {
    auto s = c.reach_right[x + 1];
    for (auto& t : c.reach_right[x + 1]) {
      QN q{std::get<0>(t), std::get<1>(t), std::get<2>(t)};
      QN r = q + c.chain.q[x];
      s.insert({r.a, r.b, r.m});
    }
    c.reach_right[x] = s;
  }
}

static const int kOpEntries[4][2][2] = {
    // {n_entries, ...} encoded as pairs (sigma_out, sigma_in); -1 = unused
    {{0, 0}, {1, 1}},     // I
    {{1, 1}, {-1, -1}},   // N
    {{1, 0}, {-1, -1}},   // C+
    {{0, 1}, {-1, -1}},   // C
};

// enlarged layout of blk with site s; left: positions 0..s (complement s+1..N-1)
static void make_layout(const Ctx& c, const SectorSet& blk, int s, bool left, Layout& lay) {
  const QN qs = c.chain.q[s];
  std::vector<QN> cand;
  for (auto& q : blk.q) {
    cand.push_back(q);
    cand.push_back(q + qs);
  }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  lay.sec.q.clear();
  lay.sec.d.clear();
  lay.pblk.clear();
  lay.poff.clear();
  const QN T = c.chain.target;
  for (auto& Q : cand) {
    bool ok = left ? reachable(c.reach_right[s + 1], T - Q) : reachable(c.reach_left[s], T - Q);
    if (!ok) continue;
    int b0 = blk.find(Q), b1 = blk.find(Q - qs);
    int d0 = b0 >= 0 ? blk.d[b0] : 0, d1 = b1 >= 0 ? blk.d[b1] : 0;
    if (d0 + d1 == 0) continue;
    lay.sec.q.push_back(Q);
    lay.sec.d.push_back(d0 + d1);
    lay.pblk.push_back({b0, b1});
    lay.poff.push_back({0, d0});
  }
}

// operators of the enlarged space (see problem.cu for the recursion); the Jordan-Wigner
// sign is (-1)^{|op| N(q_in)} on the left and (-1)^{sigma_in |O_block|} on the right.
// The host finds which blocks exist (per label, in parallel) and lays them out; the
// kernel k_enlarge assembles every block on the device.
static void ensure_site_entries(Ctx& c, int s, bool left) {
  SiteEntries& se = left ? c.ent_left[s] : c.ent_right[s];
  if (se.ready) return;
  const auto& W = c.mpo.W[s];
  const int ndst = left ? int(c.mpo.labels[s + 1].size()) : int(c.mpo.labels[s].size());
  se.ptr.assign(ndst + 1, 0);
  for (const auto& e : W) se.ptr[(left ? e.b : e.a) + 1]++;
  for (int k = 0; k < ndst; ++k) se.ptr[k + 1] += se.ptr[k];
  se.e.resize(W.size());
  std::vector<int32_t> pos(se.ptr.begin(), se.ptr.end() - 1);
  for (const auto& e : W) {   // W order inside each destination label
    EntryDev x;
    x.src = left ? e.a : e.b;
    x.op = e.op;
    x.coef = e.coef;
    se.e[pos[left ? e.b : e.a]++] = x;
  }
  se.dptr.upload(se.ptr, c.stream);
  se.de.upload(se.e, c.stream);
  se.ready = true;
}

static void ensure_dev_index(Ctx& c, OpSet& o) {
  if (o.dev_index_ready) return;
  std::vector<int64_t> boff(o.blocks.size());
  for (size_t i = 0; i < o.blocks.size(); ++i) boff[i] = o.blocks[i].off;
  std::vector<int32_t> dim(o.sec.size()), npart(o.sec.size());
  for (int i = 0; i < o.sec.size(); ++i) {
    dim[i] = o.sec.d[i];
    npart[i] = particles(o.sec.q[i]);
  }
  o.d_by_in.upload(o.by_in, c.stream);
  o.d_boff.upload(boff, c.stream);
  o.d_dim.upload(dim, c.stream);
  o.d_npart.upload(npart, c.stream);
  o.dev_index_ready = true;
}

// Persistent host worker threads (created once per process): the bookkeeping runs many
// short parallel loops per step, and starting threads for each would cost more than the
// loops.  run(nt, job) calls job(t) for t = 0..nt-1, t = 0 on the calling thread.
class WorkerPool {
 public:
  // the bookkeeping loops of one context
  static WorkerPool& get() {
    static WorkerPool pool;
    return pool;
  }
  // the instances of a batch (each instance's own loops then use get())
  static WorkerPool& instances() {
    static WorkerPool pool;
    return pool;
  }
  int size() const { return int(workers_.size()) + 1; }
  // job(t) for every t in [0, n_tasks), claimed by the workers and the calling thread.  A
  // call made while the pool is running another loop runs serially on the calling thread.
  // The first exception of a job is rethrown once every job has finished.
  void run(int n_tasks, const std::function<void(int)>& job) {
    if (n_tasks <= 0) return;
    std::unique_lock<std::mutex> caller(run_mu_, std::try_to_lock);
    if (n_tasks == 1 || workers_.empty() || !caller.owns_lock()) {
      for (int t = 0; t < n_tasks; ++t) job(t);
      return;
    }
    std::unique_lock<std::mutex> g(mu_);
    job_ = &job;
    n_tasks_ = n_tasks;
    next_ = 0;
    pending_ = n_tasks;
    error_ = nullptr;
    ++generation_;
    cv_.notify_all();
    claim(g);
    done_cv_.wait(g, [&] { return pending_ == 0; });
    job_ = nullptr;
    std::exception_ptr e = error_;
    error_ = nullptr;
    g.unlock();
    if (e) std::rethrow_exception(e);
  }

 private:
  WorkerPool() {
    const int hw = int(std::max(1u, std::thread::hardware_concurrency()));
    const int nw = std::min(16, hw) - 1;
    for (int i = 0; i < nw; ++i) workers_.emplace_back([this] { loop(); });
  }
  ~WorkerPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& w : workers_) w.join();
  }
  // run tasks of the current loop until none is left (mu_ held on entry and exit)
  void claim(std::unique_lock<std::mutex>& g) {
    while (next_ < n_tasks_) {
      const int t = next_++;
      const std::function<void(int)>* job = job_;
      g.unlock();
      std::exception_ptr e;
      try {
        (*job)(t);
      } catch (...) {
        e = std::current_exception();
      }
      g.lock();
      if (e && !error_) error_ = e;
      if (--pending_ == 0) done_cv_.notify_all();
    }
  }
  void loop() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> g(mu_);
    for (;;) {
      cv_.wait(g, [&] { return stop_ || (generation_ != seen && next_ < n_tasks_); });
      if (stop_) return;
      seen = generation_;
      claim(g);
    }
  }
  std::vector<std::thread> workers_;
  std::mutex run_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* job_ = nullptr;
  int n_tasks_ = 0, next_ = 0, pending_ = 0;
  uint64_t generation_ = 0;
  std::exception_ptr error_;
  bool stop_ = false;
};

// fn(begin, end, part) over [0, n) in up to 16 parts of at least `grain` items each; part
// p covers the p-th range in increasing order
template <class F>
static void parallel_for(int n, F&& fn, int grain = 16) {
  WorkerPool& pool = WorkerPool::get();
  int nt = std::min(pool.size(), n / std::max(1, grain));
  if (nt <= 1) {
    fn(0, n, 0);
    return;
  }
  const std::function<void(int)> job = [&](int t) {
    const int a = int(int64_t(n) * t / nt), b = int(int64_t(n) * (t + 1) / nt);
    fn(a, b, t);
  };
  pool.run(nt, job);
}

// Host part of the enlargement of blk by site s: reads the context and blk only (the site
// entries of s must be ready), so it may run on another host thread.
static void plan_enlarge(const Ctx& c, const OpSet& blk, int s, bool left, EnlPlan& P) {
  double te = wall();
  auto elap = [&](int i) {
    const double t = wall();
    P.det[i - 8] += t - te;
    te = t;
  };
  Layout& lay = P.lay;
  OpSet& out = P.out;
  make_layout(c, blk.sec, s, left, lay);
  elap(8);
  const SiteEntries& se = left ? c.ent_left[s] : c.ent_right[s];
  const int nE = lay.sec.size();
  const int nsrc = blk.sec.size();
  (void)nsrc;
  const int ndst = int(se.ptr.size()) - 1;
  const auto& dq = left ? c.mpo.dq[s + 1] : c.mpo.dq[s];
  // destination blocks (label k, Q_in) that receive at least one contribution, with
  // bitsets over the enlarged sectors: src[a][sigma] = {Q_in : source label a has a block
  // whose input sector is the piece sigma of Q_in}; ok[d][sigma] = {Q_in : Q_in + d is an
  // enlarged sector whose piece sigma exists}.  Label k gets the union over its W entries
  // of src[e.src][sigma_in] & ok[d_k][sigma_out].
  const QN qs = c.chain.q[s];
  QIndex qi_index(lay.sec);
  const int W64 = (nE + 63) / 64;
  const int nsl = blk.nlab;
  // enlarged sector of piece sigma of every source block sector
  std::vector<int32_t> piece_sec(2 * size_t(nsrc));
  for (int i = 0; i < nsrc; ++i) {
    piece_sec[2 * i] = qi_index.find(blk.sec.q[i]);
    piece_sec[2 * i + 1] = qi_index.find(blk.sec.q[i] + qs);
  }
  std::vector<uint64_t> src_bits(size_t(nsl) * 2 * W64, 0);
  parallel_for(nsl, [&](int a0, int a1, int) {
    for (int a = a0; a < a1; ++a) {
      uint64_t* bits = &src_bits[size_t(a) * 2 * W64];
      for (int64_t b = blk.lab_ptr[a]; b < blk.lab_ptr[a + 1]; ++b) {
        const int32_t* ps = &piece_sec[2 * size_t(blk.blocks[b].si)];
        if (ps[0] >= 0) bits[ps[0] / 64] |= uint64_t(1) << (ps[0] % 64);
        if (ps[1] >= 0) bits[W64 + ps[1] / 64] |= uint64_t(1) << (ps[1] % 64);
      }
    }
  });
  std::vector<QN> dk(ndst);
  for (int k = 0; k < ndst; ++k) dk[k] = left ? dq[k] : QN{0, 0, 0} - dq[k];
  std::vector<QN> dlist(dk);
  std::sort(dlist.begin(), dlist.end());
  dlist.erase(std::unique(dlist.begin(), dlist.end()), dlist.end());
  const int nd = int(dlist.size());
  std::vector<int32_t> dk_idx(ndst);
  for (int k = 0; k < ndst; ++k)
    dk_idx[k] = int32_t(std::lower_bound(dlist.begin(), dlist.end(), dk[k]) - dlist.begin());
  std::vector<uint64_t> ok_bits(size_t(nd) * 2 * W64, 0);
  std::vector<int32_t> qo_of(size_t(nd) * nE);
  parallel_for(nd, [&](int d0, int d1, int) {
    for (int di = d0; di < d1; ++di)
      for (int Qi = 0; Qi < nE; ++Qi) {
        const int Qo = qi_index.find(lay.sec.q[Qi] + dlist[di]);
        qo_of[size_t(di) * nE + Qi] = Qo;
        if (Qo < 0) continue;
        for (int sg = 0; sg < 2; ++sg)
          if (lay.pblk[Qo][sg] >= 0) ok_bits[(size_t(di) * 2 + sg) * W64 + Qi / 64] |= uint64_t(1) << (Qi % 64);
      }
  }, 2);
  elap(10);
  std::vector<std::vector<EnlBlock>>& part = P.part;
  part.assign(16, {});
  std::vector<int64_t> part_elems(16, 0);
  parallel_for(ndst, [&](int k0, int k1, int t) {
    auto& v = part[t];
    int64_t el = 0;
    std::vector<uint64_t> acc(W64);
    for (int k = k0; k < k1; ++k) {
      const size_t di = size_t(dk_idx[k]);
      std::fill(acc.begin(), acc.end(), 0);
      for (int x = se.ptr[k]; x < se.ptr[k + 1]; ++x) {
        const EntryDev& e = se.e[x];
        for (int y = 0; y < 2; ++y) {
          const int so = kOpEntries[e.op][y][0], si = kOpEntries[e.op][y][1];
          if (so < 0) continue;
          const uint64_t* sb = &src_bits[(size_t(e.src) * 2 + si) * W64];
          const uint64_t* ob = &ok_bits[(di * 2 + so) * W64];
          for (int w = 0; w < W64; ++w) acc[w] |= sb[w] & ob[w];
        }
      }
      const int32_t* qo = &qo_of[di * nE];
      for (int w = 0; w < W64; ++w)
        for (uint64_t m = acc[w]; m; m &= m - 1) {
          const int Qi = w * 64 + __builtin_ctzll(m);
          v.push_back(EnlBlock{0, k, qo[Qi], Qi, 0});
          el += (int64_t(lay.sec.d[qo[Qi]]) * lay.sec.d[Qi] + 3) & ~int64_t(3);
        }
    }
    part_elems[t] = el;
  });
  elap(11);
  // block offsets: every block starts on a 16-byte boundary (4 elements; vector loads of
  // the fused product), i.e. block b starts at the sum of the rounded-up sizes before it.
  // Threads own increasing label ranges, so concatenating their lists keeps label order.
  const int nparts = int(part.size());
  std::vector<int64_t>& pbase = P.pbase;
  pbase.assign(nparts + 1, 0);
  std::vector<int64_t> pelem(nparts + 1, 0);
  for (int t = 0; t < nparts; ++t) {
    pbase[t + 1] = pbase[t] + int64_t(part[t].size());
    pelem[t + 1] = pelem[t] + part_elems[t];
  }
  out.sec = lay.sec;
  out.nlab = ndst;
  out.lab_ptr.assign(ndst + 1, 0);
  out.blocks.resize(pbase[nparts]);
  {
    auto fill = [&](int t) {
      int64_t off = pelem[t], idx = pbase[t];
      for (EnlBlock& b : part[t]) {
        b.off = off;
        out.blocks[idx++] = OpBlock{b.Qo, b.Qi, off};
        out.lab_ptr[b.k + 1]++;   // labels of one list belong to this list only
        off += (int64_t(lay.sec.d[b.Qo]) * lay.sec.d[b.Qi] + 3) & ~int64_t(3);
      }
    };
    WorkerPool::get().run(nparts, [&](int t) { fill(t); });
  }
  for (int k = 0; k < ndst; ++k) out.lab_ptr[k + 1] += out.lab_ptr[k];
  out.n_elems = pelem[nparts];
  elap(12);
  // device tables and the index by input sector (host)
  P.ld.resize(nE);
  for (int i = 0; i < nE; ++i)
    P.ld[i] = LayDev{lay.pblk[i][0], lay.pblk[i][1], lay.poff[i][1], lay.sec.d[i]};
  out.index_by_in();
  elap(14);
}

// Device part: the arena, the tables, the kernel.  Without `ahead`: on the context stream,
// waited for.  With `ahead`: on the prefetch stream after the context stream's work so far,
// not waited for; the tables are kept in `ahead` until the result is used.
static void exec_enlarge(Ctx& c, OpSet& blk, int s, bool left, EnlPlan& P, Layout& lay,
                         OpSet& out, Prefetch* ahead = nullptr) {
  double te = wall();
  ensure_dev_index(c, blk);
  c.t_detail[9] += wall() - te;
  const SiteEntries& se = left ? c.ent_left[s] : c.ent_right[s];
  lay = std::move(P.lay);
  out = std::move(P.out);
  out.data.alloc(out.n_elems + 4);
  cudaStream_t st = c.stream;
  if (ahead) {
    if (!ahead->st) {
      DMRG_CUDA(cudaStreamCreateWithFlags(&ahead->st, cudaStreamNonBlocking));
      DMRG_CUDA(cudaEventCreateWithFlags(&ahead->ready, cudaEventDisableTiming));
      DMRG_CUDA(cudaEventCreateWithFlags(&ahead->done, cudaEventDisableTiming));
    }
    // pool memory handed out above may still be in use by earlier work on the context stream
    DMRG_CUDA(cudaEventRecord(ahead->ready, c.stream));
    DMRG_CUDA(cudaStreamWaitEvent(ahead->st, ahead->ready, 0));
    st = ahead->st;
  }
  const int nparts = int(P.part.size());
  DevBuf<LayDev> dlay;
  DevBuf<EnlBlock> deb;
  dlay.upload(P.ld, st);
  deb.alloc(std::max<int64_t>(P.pbase[nparts], 1));
  for (int t = 0; t < nparts; ++t)
    if (!P.part[t].empty())
      DMRG_CUDA(cudaMemcpyAsync(deb.p + P.pbase[t], P.part[t].data(),
                                sizeof(EnlBlock) * P.part[t].size(), cudaMemcpyHostToDevice, st));
  const int64_t n_eb = P.pbase[nparts];
  const auto& spar = left ? c.mpo.parity[s] : c.mpo.parity[s + 1];
  DevBuf<int8_t> dpar;
  dpar.upload(spar, st);
  enlarge_blocks(deb.p, n_eb, se.dptr.p, se.de.p, blk.d_by_in.p, blk.sec.size(), blk.d_boff.p,
                 blk.d_dim.p, blk.d_npart.p, dpar.p, dlay.p, left ? 1 : 0, blk.data.p,
                 out.data.p, st);
  if (ahead) {
    DMRG_CUDA(cudaEventRecord(ahead->done, st));
    ahead->t_lay = std::move(dlay);
    ahead->t_blocks = std::move(deb);
    ahead->t_par = std::move(dpar);
    return;
  }
  te = wall();
  sync(c);   // the small tables above are released
  c.t_detail[7] += wall() - te;
}

static void wait_prefetch(Ctx& c) {
  if (c.pf.th.joinable()) c.pf.th.join();
}

// a finished plan for (blk, s, left) if one was prefetched
// the enlarged set issued ahead for (blk, s, left), made visible to the context stream
static bool take_prefetch_device(Ctx& c, uint64_t gen, int s, bool left, Layout& lay,
                                 OpSet& out) {
  if (!c.pf.dev_ready || c.pf.s != s || c.pf.left != left) return false;
  c.pf.dev_ready = false;
  c.pf.active = false;
  DMRG_CUDA(cudaStreamWaitEvent(c.stream, c.pf.done, 0));
  // the tables go back to the pool once the context stream is past the kernel
  c.pf.t_lay.release();
  c.pf.t_blocks.release();
  c.pf.t_par.release();
  if (c.pf.gen != gen) {   // stale (cannot happen within a sweep): drop it
    c.pf.out = OpSet();
    return false;
  }
  lay = std::move(c.pf.lay);
  out = std::move(c.pf.out);
  return true;
}

static bool take_prefetch(Ctx& c, uint64_t gen, int s, bool left, EnlPlan& P) {
  if (!c.pf.active || c.pf.dev_ready || c.pf.s != s || c.pf.left != left) return false;
  wait_prefetch(c);
  c.pf.active = false;
  const bool hit = !c.pf.err && c.pf.s == s && c.pf.left == left && c.pf.gen == gen;
  if (hit) P = std::move(c.pf.plan);
  c.pf.plan = EnlPlan();
  c.pf.err = nullptr;
  return hit;
}

// plan the enlargement of blk by site s on a host thread (gen: blk's generation)
static void start_prefetch(Ctx& c, const OpSet& blk, uint64_t gen, int s, bool left) {
  wait_prefetch(c);
  if (c.pf.dev_ready) {   // an unused result: drop it once its kernel is done
    DMRG_CUDA(cudaStreamSynchronize(c.pf.st));
    c.pf.dev_ready = false;
    c.pf.out = OpSet();
    c.pf.t_lay.release();
    c.pf.t_blocks.release();
    c.pf.t_par.release();
  }
  ensure_site_entries(c, s, left);   // main thread: may upload
  c.pf.active = true;
  c.pf.s = s;
  c.pf.left = left;
  c.pf.gen = gen;
  c.pf.plan = EnlPlan();
  c.pf.err = nullptr;
  const Ctx* cc = &c;
  const OpSet* src = &blk;
  Prefetch* pf = &c.pf;
  c.pf.th = std::thread([cc, src, s, left, pf] {
    try {
      plan_enlarge(*cc, *src, s, left, pf->plan);
    } catch (...) {
      pf->err = std::current_exception();
    }
  });
}

// once its plan is made, issue the prefetched enlargement on the prefetch stream (called
// while the context stream is nearly idle: after Davidson)
static void issue_prefetch_device(Ctx& c, OpSet& blk) {
  if (!c.pf.active || c.pf.dev_ready) return;
  wait_prefetch(c);
  if (c.pf.err) return;
  c.pf.active = false;   // the plan is consumed; restored once the launch is issued
  exec_enlarge(c, blk, c.pf.s, c.pf.left, c.pf.plan, c.pf.lay, c.pf.out, &c.pf);
  c.pf.plan = EnlPlan();
  c.pf.active = true;
  c.pf.dev_ready = true;
}

// operators of the enlarged space; blk_gen identifies blk for a prefetched plan (0: none)
static void enlarge(Ctx& c, OpSet& blk, int s, bool left, Layout& lay, OpSet& out,
                    uint64_t blk_gen = 0) {
  PhaseTimer tm(c.t_enlarge);
  if (blk_gen && take_prefetch_device(c, blk_gen, s, left, lay, out)) return;
  const double th0 = wall();
  EnlPlan P;
  if (!(blk_gen && take_prefetch(c, blk_gen, s, left, P))) {
    ensure_site_entries(c, s, left);
    plan_enlarge(c, blk, s, left, P);
    for (int i = 0; i < 8; ++i) c.t_detail[8 + i] += P.det[i];
  }
  c.t_enlarge_host += wall() - th0;
  exec_enlarge(c, blk, s, left, P, lay, out);
}

// stored block = kept part of an enlarged operator set: O' = U_o^T O U_i per block
static void project(Ctx& c, OpSet& E, const Iso& iso, OpSet& out) {
  PhaseTimer tm(c.t_project);
  if (iso.identity) {
    out = std::move(E);   // its index by input sector was built with it
    out.dev_index_ready = false;
    return;
  }
  const int nE = E.sec.size();
  out.sec.q.clear();
  out.sec.d.clear();
  for (int i = 0; i < nE; ++i)
    if (iso.m[i] > 0) {
      out.sec.q.push_back(E.sec.q[i]);
      out.sec.d.push_back(iso.m[i]);
    }
  out.nlab = E.nlab;
  out.lab_ptr.assign(E.nlab + 1, 0);
  out.blocks.clear();
  double tp = wall();
  // one renormalization task per kept block, read by k_project straight from this table
  std::vector<ProjTask> tasks, small;
  small.reserve(E.blocks.size());
  std::vector<int64_t> tb1(1, 0), tb2(1, 0);
  int64_t noff = 0, toff = 0;
  for (int k = 0; k < E.nlab; ++k) {
    out.lab_ptr[k] = int64_t(out.blocks.size());
    for (int64_t x = E.lab_ptr[k]; x < E.lab_ptr[k + 1]; ++x) {
      const OpBlock& b = E.blocks[x];
      const int no = iso.kept_idx[b.so], ni = iso.kept_idx[b.si];
      if (no < 0 || ni < 0) continue;
      const int Do = E.sec.d[b.so], Di = E.sec.d[b.si], mo = iso.m[b.so], mi = iso.m[b.si];
      DMRG_REQUIRE(b.off + int64_t(Do) * Di <= E.n_elems, DMRG_EINVAL,
                   "internal: operator block out of range");
      out.blocks.push_back(OpBlock{no, ni, noff});
      if (Do <= 32 && Di <= 32) {
        small.push_back(ProjTask{b.off, noff, 0, b.so, b.si});
      } else {
        tasks.push_back(ProjTask{b.off, noff, toff, b.so, b.si});
        const int64_t ct = (mi + 31) / 32;
        tb1.push_back(tb1.back() + (Do + 31) / 32 * ct);
        tb2.push_back(tb2.back() + (mo + 31) / 32 * ct);
        toff += int64_t(Do) * mi;
      }
      noff += int64_t(mo) * mi;
    }
  }
  out.lab_ptr[E.nlab] = int64_t(out.blocks.size());
  out.n_elems = noff;
  std::vector<int64_t> uo(nE);
  for (int i = 0; i < nE; ++i) {
    uo[i] = iso.uoff[i];
    DMRG_REQUIRE(iso.m[i] == 0 || uo[i] + int64_t(E.sec.d[i]) * iso.m[i] <= iso.data.n,
                 DMRG_EINVAL, "internal: isometry out of range");
  }
  out.data.alloc(std::max<int64_t>(noff, 1));
  c.tmp.alloc(std::max<int64_t>(toff, 1));
  DevBuf<ProjTask> dt, dts;
  DevBuf<int32_t> dD, dm;
  DevBuf<int64_t> duo, dtb1, dtb2;
  dt.upload(tasks, c.stream);
  dts.upload(small, c.stream);
  dtb1.upload(tb1, c.stream);
  dtb2.upload(tb2, c.stream);
  dD.upload(E.sec.d, c.stream);
  dm.upload(iso.m, c.stream);
  duo.upload(uo, c.stream);
  c.t_detail[4] += wall() - tp;
  tp = wall();
  project_small(dts.p, int64_t(small.size()), dD.p, dm.p, duo.p, E.data.p, iso.data.p,
                out.data.p, c.stream);
  // FP64 in both precisions: the stored operators must keep the Hermitian pairing of the
  // normal and complementary operators to FP64 rounding; split-TF32 products left the pairs
  // unequal at ~1e-6 relative, which floored the Davidson residual of the next steps
  project_blocks(dt.p, dtb1.p, tb1.back(), dtb2.p, tb2.back(), int64_t(tasks.size()), dD.p,
                 dm.p, duo.p, E.data.p, iso.data.p, c.tmp.p, out.data.p, c.stream);
  sync(c);
  c.t_detail[5] += wall() - tp;
  tp = wall();
  out.index_by_in();
  c.t_detail[6] += wall() - tp;
}

static void identity_iso(Ctx& c, const Layout& lay, Iso& iso) {
  iso.lay = lay;
  const int n = lay.sec.size();
  iso.m = lay.sec.d;
  iso.uoff.assign(n, 0);
  iso.kept_idx.resize(n);
  iso.enl_idx.resize(n);
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    iso.kept_idx[i] = i;
    iso.enl_idx[i] = i;
    iso.uoff[i] = off;
    off += int64_t(lay.sec.d[i]) * lay.sec.d[i];
  }
  // zeros, then ones at the diagonal positions (built on the device)
  std::vector<int64_t> diag;
  diag.reserve(size_t(lay.sec.total()));
  for (int i = 0; i < n; ++i)
    for (int r = 0; r < lay.sec.d[i]; ++r) diag.push_back(iso.uoff[i] + int64_t(r) * lay.sec.d[i] + r);
  iso.data.alloc(std::max<int64_t>(off, 1));
  DMRG_CUDA(cudaMemsetAsync(iso.data.p, 0, sizeof(double) * std::max<int64_t>(off, 1), c.stream));
  DevBuf<int64_t> dd;
  dd.upload(diag, c.stream);
  set_ones(iso.data.p, dd.p, int64_t(diag.size()), c.stream);
  sync(c);   // dd is released
  iso.identity = true;
}

static void finish_iso_index(Iso& iso) {
  const int n = iso.lay.sec.size();
  iso.kept_idx.assign(n, -1);
  iso.enl_idx.clear();
  for (int i = 0; i < n; ++i)
    if (iso.m[i] > 0) {
      iso.kept_idx[i] = int(iso.enl_idx.size());
      iso.enl_idx.push_back(i);
    }
}

static OpSet vacuum_ops(int nlab, int which, cudaStream_t s) {
  OpSet v;
  v.sec.q = {QN{0, 0, 0}};
  v.sec.d = {1};
  v.nlab = nlab;
  v.lab_ptr.assign(nlab + 1, 0);
  for (int k = which + 1; k <= nlab; ++k) v.lab_ptr[k] = 1;
  v.blocks = {OpBlock{0, 0, 0}};
  double one = 1.0;
  v.data.upload(&one, 1, s);
  v.n_elems = 1;
  v.index_by_in();
  return v;
}

// ---------------------------------------------------------------------------------------
// superblock at position p: enlarged operators, wave-function layout, H_eff task lists
// ---------------------------------------------------------------------------------------
static void build_super(Ctx& c, int p) {
  PhaseTimer tm(c.t_super);
  DMRG_REQUIRE(c.built, DMRG_EINVAL, "dmrg_build_blocks has not been called");
  DMRG_REQUIRE(p >= 1 && p <= c.N - 3, DMRG_EINVAL, "position out of range [1, N-3]");
  DMRG_REQUIRE(c.left[p - 1].valid && c.right[p + 1].valid, DMRG_EINVAL,
               "blocks for this position are not available");
  auto sb = std::make_unique<Super>();
  sb->p = p;
  enlarge(c, c.left[p - 1].ops, p, true, sb->Ll, sb->L, c.left[p - 1].gen);
  enlarge(c, c.right[p + 1].ops, p + 1, false, sb->Rl, sb->R, c.right[p + 1].gen);
  const QN T = c.chain.target;
  const int nL = sb->Ll.sec.size(), nR = sb->Rl.sec.size();
  sb->psi_of_L.assign(nL, -1);
  sb->psi_of_R.assign(nR, -1);
  int64_t off = 0;
  for (int i = 0; i < nL; ++i) {
    int j = sb->Rl.sec.find(T - sb->Ll.sec.q[i]);
    if (j < 0) continue;
    sb->psi_of_L[i] = int(sb->bL.size());
    sb->psi_of_R[j] = int(sb->bL.size());
    sb->bL.push_back(i);
    sb->bR.push_back(j);
    sb->bdl.push_back(sb->Ll.sec.d[i]);
    sb->bdr.push_back(sb->Rl.sec.d[j]);
    sb->boff.push_back(off);
    off += int64_t(sb->Ll.sec.d[i]) * sb->Rl.sec.d[j];
  }
  sb->size = off;
  {
    int64_t po = 0;
    std::vector<int32_t> len(sb->bL.size());
    for (size_t b = 0; b < sb->bL.size(); ++b) {
      po = (po + 3) & ~int64_t(3);
      sb->pad_off.push_back(po);
      len[b] = sb->bdl[b] * sb->bdr[b];
      po += len[b];
    }
    sb->pad_size = po + 4;
    sb->d_src_off.upload(sb->boff, c.stream);
    sb->d_pad_off.upload(sb->pad_off, c.stream);
    sb->d_pad_len.upload(len, c.stream);
  }
  double tp = wall();
  auto lap = [&](int i) {
    const double t = wall();
    c.t_detail[i] += t - tp;
    tp = t;
  };
  // H_eff terms (label k, L block, R block) per output block, in label order; built in
  // parallel over output blocks (the L block of label k into output sector Q has input
  // sector Q - dq_k)
  const auto& par = c.mpo.parity[p + 1];
  const auto& dqL = c.mpo.dq[p + 1];
  const int nlab = sb->L.nlab;
  DMRG_REQUIRE(nlab == sb->R.nlab, DMRG_EINVAL, "internal: label count mismatch");
  struct Item {
    int64_t lb, rb;
    int bin, bout;
    double sign;
  };
  const int nb = int(sb->bL.size());
  QIndex qL(sb->Ll.sec);
  std::vector<std::vector<Item>> by_out(nb);
  std::atomic<bool> broken{false};
  parallel_for(nb, [&](int b0, int b1, int) {
    for (int bo = b0; bo < b1; ++bo) {
      const int so = sb->bL[bo];
      auto& v = by_out[bo];
      for (int k = 0; k < nlab; ++k) {
        const int si = qL.find(sb->Ll.sec.q[so] - dqL[k]);
        if (si < 0) continue;
        const int bin = sb->psi_of_L[si];
        if (bin < 0) continue;
        const int lb = sb->L.by_in[size_t(k) * nL + si];
        if (lb < 0) continue;
        const int rb = sb->R.by_in[size_t(k) * nR + sb->bR[bin]];
        if (rb < 0) continue;
        if (sb->L.blocks[lb].so != so || sb->R.blocks[rb].so != sb->bR[bo]) broken = true;
        const double sign = (par[k] && (particles(sb->Ll.sec.q[si]) & 1)) ? -1.0 : 1.0;
        v.push_back(Item{lb, rb, bin, bo, sign});
      }
    }
  });
  DMRG_REQUIRE(!broken, DMRG_EINVAL, "internal: superblock term breaks the target sector");
  lap(0);
  // fused product: items grouped by output block, output tiles of at most 32 x 32, groups
  // of at most G terms per thread block (partial tiles summed in group order); counts per
  // output block first, then every block fills its own ranges in parallel
  // small output blocks (every dimension of the block and of its terms <= kSmallEdge) are
  // single tiles of the warp kernel with groups of at most Gs terms
  const int G = 64, Gs = 16;
  std::vector<int64_t> i_beg(nb + 1, 0), t_beg(nb + 1, 0), s_beg(nb + 1, 0), r_beg(nb + 1, 0),
      p_beg(nb + 1, 0);
  std::vector<char> small_bo(nb, 0), big_bo(nb, 0);
  for (int bo = 0; bo < nb; ++bo) {
    const int ni = int(by_out[bo].size());
    bool sm = sb->bdl[bo] <= kSmallEdge && sb->bdr[bo] <= kSmallEdge;
    int wide = std::max(sb->bdl[bo], sb->bdr[bo]);
    for (int j = 0; j < ni; ++j) {
      const int bin = by_out[bo][j].bin;
      sm = sm && sb->bdl[bin] <= kSmallEdge && sb->bdr[bin] <= kSmallEdge;
      wide = std::max(wide, std::max(sb->bdl[bin], sb->bdr[bin]));
    }
    small_bo[bo] = sm;
    const bool big = !sm && c.big_edge > 0 && wide > c.big_edge;
    big_bo[bo] = big;
    const int groups = sm ? std::max(1, (ni + Gs - 1) / Gs) : std::max(1, (ni + G - 1) / G);
    const int64_t tiles = sm ? 1 : int64_t((sb->bdl[bo] + 31) / 32) * ((sb->bdr[bo] + 31) / 32);
    i_beg[bo + 1] = i_beg[bo] + ni;
    t_beg[bo + 1] = t_beg[bo] + (sm || big ? 0 : tiles * groups);
    s_beg[bo + 1] = s_beg[bo] + (sm ? groups : 0);
    r_beg[bo + 1] = r_beg[bo] + (groups > 1 && !big ? tiles : 0);
    p_beg[bo + 1] = p_beg[bo] + (groups > 1 && !big ? int64_t(groups) * sb->bdl[bo] * sb->bdr[bo] : 0);
  }
  DMRG_REQUIRE(i_beg[nb] < (int64_t(1) << 31), DMRG_EINVAL, "superblock has too many terms");
  struct TileCost {
    HeffTile t;
    double cost;
  };
  std::vector<HeffItem> fi(i_beg[nb]);
  std::vector<TileCost> ft(t_beg[nb]), fts(s_beg[nb]);
  std::vector<HeffRed> fr(r_beg[nb]);
  std::vector<double> bo_flops(nb, 0.0), bo_bytes(nb, 0.0), bo_kflops(nb, 0.0);
  std::vector<int64_t> bo_toff(nb, 0);
  std::vector<std::array<double, 8>> bo_hist(nb);
  sb->terms_host.resize(i_beg[nb]);
  parallel_for(nb, [&](int b0, int b1, int) {
    for (int bo = b0; bo < b1; ++bo) {
      const int dLo = sb->bdl[bo], dRo = sb->bdr[bo];
      const int i0 = int(i_beg[bo]), i1 = int(i_beg[bo + 1]);
      double work = 0, fl = 0, by = 0, kfl = 0;
      std::array<double, 8> hist{};
      int64_t to = 0;
      for (int j = i0; j < i1; ++j) {
        const Item& it = by_out[bo][j - i0];
        const int dLi = sb->bdl[it.bin], dRi = sb->bdr[it.bin];
        HeffItem& h = fi[j];
        h.loff = sb->L.blocks[it.lb].off;
        h.roff = sb->R.blocks[it.rb].off;
        h.xoff = sb->pad_off[it.bin];
        h.dLi = dLi;
        h.dRi = dRi;
        h.sign = float(it.sign);
        h.pad = 0;
        work += double(dLi) * dRi + double(dLi);
        to += int64_t(dLi) * dRo;
        const double f1 = 2.0 * dLi * dRi * dRo + 2.0 * dLo * dLi * dRo;
        const double f2 = 2.0 * dLo * dLi * dRi + 2.0 * dLo * dRi * dRo;
        fl += std::min(f1, f2);
        // an L block (label, input sector) and an R block each belong to one term only
        by += double(dLo) * dLi + double(dRo) * dRi;
        const int dmax = std::max(dLi, dRi);
        const int cls = dmax <= 8 ? 0 : dmax <= 16 ? 1 : dmax <= 32 ? 2 : 3;
        hist[cls] += 1.0;
        hist[4 + cls] += std::min(f1, f2);
        // the tile kernels form psi R^T first; the grouped passes take the cheaper order
        kfl += big_bo[bo] ? std::min(f1, f2) : f1;
        sb->terms_host[j] = Super::Term{it.lb, it.rb, it.bin, it.bout, it.sign};
      }
      bo_flops[bo] = fl;
      bo_kflops[bo] = kfl;
      bo_bytes[bo] = by;
      bo_hist[bo] = hist;
      bo_toff[bo] = to;
      if (big_bo[bo]) continue;   // the grouped GEMM passes below
      const bool sm = small_bo[bo];
      const int GG = sm ? Gs : G, edge = sm ? kSmallEdge : 32;
      const int groups = std::max(1, (i1 - i0 + GG - 1) / GG);
      int64_t tpos = sm ? s_beg[bo] : t_beg[bo], rpos = r_beg[bo], pelems = p_beg[bo];
      std::vector<TileCost>& dst = sm ? fts : ft;
      for (int r0 = 0; r0 < dLo; r0 += edge)
        for (int c0 = 0; c0 < dRo; c0 += edge) {
          HeffTile t;
          t.yoff = sb->boff[bo];
          t.ld = dRo;
          t.r0 = r0;
          t.c0 = c0;
          t.m = std::min(edge, dLo - r0);
          t.n = std::min(edge, dRo - c0);
          t.inst = 0;
          const int64_t mn = int64_t(t.m) * t.n;
          if (groups > 1) {
            HeffRed rd;
            rd.yoff = t.yoff;
            rd.poff = pelems;
            rd.ld = t.ld;
            rd.r0 = r0;
            rd.c0 = c0;
            rd.m = t.m;
            rd.n = t.n;
            rd.groups = groups;
            rd.inst = 0;
            rd.pad = 0;
            fr[rpos++] = rd;
          }
          for (int g = 0; g < groups; ++g) {
            t.i0 = i0 + g * GG;
            t.i1 = std::min(i1, t.i0 + GG);
            t.poff = groups > 1 ? pelems + g * mn : -1;
            dst[tpos++] = TileCost{t, work * double(t.i1 - t.i0) / std::max(1, i1 - i0) * t.n + 1.0};
          }
          if (groups > 1) pelems += groups * mn;
        }
    }
  });
  int64_t toff = 0;
  double flops = 0, bytes = 0;
  std::array<double, 8> hist{};
  for (int bo = 0; bo < nb; ++bo) {
    flops += bo_flops[bo];
    bytes += bo_bytes[bo];
    toff += bo_toff[bo];
    for (int i = 0; i < 8; ++i) hist[i] += bo_hist[bo][i];
  }
  for (int i = 0; i < 8; ++i) c.term_hist[i] = int64_t(hist[i]);
  c.kernel_flops = 0;
  for (int bo = 0; bo < nb; ++bo) c.kernel_flops += bo_kflops[bo];
  const int64_t items = i_beg[nb];
  const int64_t pelems = p_beg[nb];
  sb->t_elems = toff;
  sb->n_items = items;
  c.last_sizes[0] = int64_t(sb->L.blocks.size());
  c.last_sizes[1] = int64_t(sb->R.blocks.size());
  c.last_sizes[2] = items;
  c.last_sizes[3] = int64_t(ft.size());
  c.last_sizes[4] = int64_t(fts.size());
  sb->flops = flops;
  bytes += 2.0 * double(sb->size);
  sb->bytes = bytes * (c.opt.precision == DMRG_FP64 ? 8.0 : 4.0);
  lap(1);
  {
    // heaviest tiles first; validate every access range on the host
    auto by_cost = [](const TileCost& a, const TileCost& b) { return a.cost > b.cost; };
    std::stable_sort(ft.begin(), ft.end(), by_cost);
    std::stable_sort(fts.begin(), fts.end(), by_cost);
    auto check = [&](const std::vector<TileCost>& v, std::vector<HeffTile>& tl, int edge) {
      tl.resize(v.size());
      for (size_t i = 0; i < v.size(); ++i) {
        const HeffTile& t = v[i].t;
        tl[i] = t;
        DMRG_REQUIRE(t.m >= 1 && t.n >= 1 && t.m <= edge && t.n <= edge &&
                         t.yoff + int64_t(t.r0 + t.m - 1) * t.ld + t.c0 + t.n - 1 < sb->size,
                     DMRG_EINVAL, "internal: fused tile out of range");
        for (int j = t.i0; j < t.i1; ++j) {
          const HeffItem& h = fi[j];
          DMRG_REQUIRE(h.loff + int64_t(t.r0 + t.m) * h.dLi - 1 < sb->L.n_elems &&
                           h.roff + int64_t(t.c0 + t.n) * h.dRi - 1 < sb->R.n_elems &&
                           h.xoff + int64_t(h.dLi) * h.dRi - 1 < sb->pad_size - 4 &&
                           (edge == 32 || (h.dLi <= kSmallEdge && h.dRi <= kSmallEdge)),
                       DMRG_EINVAL, "internal: fused item out of range");
        }
      }
    };
    std::vector<HeffTile> tl, tls;
    check(ft, tl, 32);
    check(fts, tls, kSmallEdge);
    for (const HeffRed& r : fr)
      DMRG_REQUIRE(r.poff + int64_t(r.groups) * r.m * r.n <= pelems &&
                       r.yoff + int64_t(r.r0 + r.m - 1) * r.ld + r.c0 + r.n - 1 < sb->size,
                   DMRG_EINVAL, "internal: partial tile out of range");
    sb->fitems.upload(fi, c.stream);
    sb->ftiles.upload(tl, c.stream);
    sb->stiles.upload(tls, c.stream);
    sb->fred.upload(fr, c.stream);
    // host copies for batch mode (lists of several instances in one launch)
    sb->h_items = std::move(fi);
    sb->h_tiles = std::move(tl);
    sb->h_stiles = std::move(tls);
    sb->h_red = std::move(fr);
    sb->h_cost.resize(ft.size());
    for (size_t i = 0; i < ft.size(); ++i) sb->h_cost[i] = ft[i].cost;
    sb->h_scost.resize(fts.size());
    for (size_t i = 0; i < fts.size(); ++i) sb->h_scost[i] = fts[i].cost;
    sb->n_ftiles = int64_t(sb->h_tiles.size());
    sb->n_stiles = int64_t(sb->h_stiles.size());
    sb->n_fred = int64_t(sb->h_red.size());
    sb->p_elems = pelems;
  }
  {
    // grouped GEMM passes of the big output blocks, each term in its cheaper association:
    // T = psi R^T then s L T, or Z = L psi then s Z R^T (both kinds of terms may share a
    // stage-2 task).  Stage 2 sums over every term of an output block (K = sum of the
    // terms' inner dimensions, tens of thousands at M = 4096), so the terms
    // are cut into groups of at most kBigGroupK inner elements: each group writes a partial
    // block, and the partial blocks are added in group order afterwards (deterministic)
    constexpr int64_t kBigGroupK = 2048;
    TaskList g1, g2;
    std::vector<HeffRed> red2;
    int64_t toff2 = 0, poff2 = 0;
    for (int bo = 0; bo < nb; ++bo) {
      if (!big_bo[bo]) continue;
      ++sb->n_big_blocks;
      const int dLo = sb->bdl[bo], dRo = sb->bdr[bo];
      const int64_t mn = int64_t(dLo) * dRo;
      // groups of terms
      std::vector<int64_t> gstart(1, i_beg[bo]);
      int64_t kacc = 0;
      for (int64_t j = i_beg[bo]; j < i_beg[bo + 1]; ++j) {
        const int dLi = sb->bdl[sb->terms_host[j].bin], dRi = sb->bdr[sb->terms_host[j].bin];
        const double f1 = 2.0 * dLi * dRi * dRo + 2.0 * dLo * dLi * dRo;
        const double f2 = 2.0 * dLo * dLi * dRi + 2.0 * dLo * dRi * dRo;
        const int kk = f1 <= f2 ? dLi : dRi;   // the inner dimension of its stage-2 term
        if (kacc > 0 && kacc + kk > kBigGroupK) {
          gstart.push_back(j);
          kacc = 0;
        }
        kacc += kk;
      }
      gstart.push_back(i_beg[bo + 1]);
      const int groups = int(gstart.size()) - 1;
      for (int g = 0; g < groups; ++g) {
        if (groups == 1) g2.begin_task(Operand{sb->boff[bo], B_Y, dRo}, dLo, dRo);
        else g2.begin_task(Operand{poff2 + g * mn, B_Z, dRo}, dLo, dRo);
        for (int64_t j = gstart[g]; j < gstart[g + 1]; ++j) {
          const Super::Term& tm = sb->terms_host[j];
          const int dLi = sb->bdl[tm.bin], dRi = sb->bdr[tm.bin];
          // the cheaper association of L psi R^T for this term
          const double f1 = 2.0 * dLi * dRi * dRo + 2.0 * dLo * dLi * dRo;   // psi R^T first
          const double f2 = 2.0 * dLo * dLi * dRi + 2.0 * dLo * dRi * dRo;   // L psi first
          if (f1 <= f2) {
            // T = psi R^T (d_Li x d_Ro), then psi' += s L T
            g1.begin_task(Operand{toff2, B_T, dRo}, dLi, dRo);
            g1.add_term(Operand{sb->pad_off[tm.bin], B_X, dRi},
                        Operand{sb->R.blocks[tm.rb].off, B_ROPS, dRi}, dRi, 2, 1.0);
            g2.add_term(Operand{sb->L.blocks[tm.lb].off, B_LOPS, dLi},
                        Operand{toff2, B_T, dRo}, dLi, 0, tm.sign);
            toff2 += int64_t(dLi) * dRo;
          } else {
            // Z = L psi (d_Lo x d_Ri), then psi' += s Z R^T
            g1.begin_task(Operand{toff2, B_T, dRi}, dLo, dRi);
            g1.add_term(Operand{sb->L.blocks[tm.lb].off, B_LOPS, dLi},
                        Operand{sb->pad_off[tm.bin], B_X, dRi}, dLi, 0, 1.0);
            g2.add_term(Operand{toff2, B_T, dRi}, Operand{sb->R.blocks[tm.rb].off, B_ROPS, dRi},
                        dRi, 2, tm.sign);
            toff2 += int64_t(dLo) * dRi;
          }
        }
      }
      if (groups > 1) {
        HeffRed r;
        r.yoff = sb->boff[bo];
        r.poff = poff2;
        r.ld = dRo;
        r.r0 = 0;
        r.c0 = 0;
        r.m = dLo;
        r.n = dRo;
        r.groups = groups;
        r.inst = 0;
        r.pad = 0;
        red2.push_back(r);
        poff2 += int64_t(groups) * mn;
      }
    }
    sb->big_t_elems = toff2;
    sb->big_p_elems = poff2;
    if (sb->n_big_blocks) {
      int64_t be[NBASE] = {0};
      be[B_X] = sb->pad_size;
      be[B_Y] = sb->size;
      be[B_T] = std::max<int64_t>(toff2, 1);
      be[B_Z] = std::max<int64_t>(poff2, 1);
      be[B_LOPS] = sb->L.n_elems;
      be[B_ROPS] = sb->R.n_elems;
      // the tensor-core engine takes every task as tiles; the FP64 one runs small tasks
      // one warp each
      const int64_t lim = c.opt.precision == DMRG_FP64 ? 1024 : 0;
      sb->big1.build(g1, be, c.stream, lim);
      sb->big2.build(g2, be, c.stream, lim);
      sb->big_red.upload(red2, c.stream);
      sb->n_big_red = int64_t(red2.size());
    }
  }
  lap(2);
  // diagonal tasks: terms that keep the sector (Delta q = 0)
  std::vector<DiagTask> dt;
  std::vector<DiagTerm> dg;
  std::vector<int> diag_labels;
  for (int k = 0; k < nlab; ++k) {
    const QN& d = c.mpo.dq[p + 1][k];
    if (d.a == 0 && d.b == 0 && d.m == 0) diag_labels.push_back(k);
  }
  for (size_t b = 0; b < sb->bL.size(); ++b) {
    DiagTask t;
    t.psi_off = sb->boff[b];
    t.dL = sb->bdl[b];
    t.dR = sb->bdr[b];
    t.t0 = int(dg.size());
    for (int k : diag_labels) {
      int lb = sb->L.by_in[size_t(k) * nL + sb->bL[b]];
      int rb = sb->R.by_in[size_t(k) * nR + sb->bR[b]];
      if (lb < 0 || rb < 0) continue;
      dg.push_back(DiagTerm{sb->L.blocks[lb].off, sb->R.blocks[rb].off, t.dL, t.dR});
    }
    t.t1 = int(dg.size());
    dt.push_back(t);
  }
  sb->dtasks.upload(dt, c.stream);
  sb->dterms.upload(dg, c.stream);
  sb->n_dtasks = int(dt.size());
  lap(3);
  if (c.opt.precision != DMRG_FP64) {
    sb->L.data32.alloc(sb->L.n_elems + 4);
    sb->R.data32.alloc(sb->R.n_elems + 4);
    to_f32(sb->L.data.p, sb->L.data32.p, sb->L.n_elems, c.stream);
    to_f32(sb->R.data.p, sb->R.data32.p, sb->R.n_elems, c.stream);
  }
  sync(c);
  c.sb = std::move(sb);
}

static Super& super_at(Ctx& c, int p) {
  if (!c.sb || c.sb->p != p) build_super(c, p);
  return *c.sb;
}

// two-stage H_eff lists (T = psi R^T, then psi' = sum s L T) used by the allocation-free
// entry point; built by the allocating ABI calls only
static void ensure_two_stage(Ctx& c, Super& sb) {
  // only superblocks whose intermediate fits the allocation-free product's array need them
  if (sb.two_stage_ready || sb.t_elems > kScratchElems) return;
  TaskList s1, s2;
  int64_t toff = 0;
  int last_out = -1;
  for (const auto& it : sb.terms_host) {
    const int dLi = sb.bdl[it.bin], dRi = sb.bdr[it.bin];
    const int dLo = sb.bdl[it.bout], dRo = sb.bdr[it.bout];
    if (it.bout != last_out) {
      s2.begin_task(Operand{sb.boff[it.bout], B_Y, dRo}, dLo, dRo);
      last_out = it.bout;
    }
    s1.begin_task(Operand{toff, B_T, dRo}, dLi, dRo);
    s1.add_term(Operand{sb.boff[it.bin], B_X, dRi}, Operand{sb.R.blocks[it.rb].off, B_ROPS, dRi},
                dRi, 2, 1.0);
    s2.add_term(Operand{sb.L.blocks[it.lb].off, B_LOPS, dLi}, Operand{toff, B_T, dRo}, dLi, 0,
                it.sign);
    toff += int64_t(dLi) * dRo;
  }
  DMRG_REQUIRE(toff == sb.t_elems, DMRG_EINVAL, "internal: two-stage intermediate size");
  int64_t be[NBASE] = {0};
  be[B_X] = sb.size;
  be[B_Y] = sb.size;
  be[B_T] = sb.t_elems;
  be[B_LOPS] = sb.L.n_elems;
  be[B_ROPS] = sb.R.n_elems;
  sb.st1.build(s1, be, c.stream);
  sb.st2.build(s2, be, c.stream);
  sync(c);
  sb.two_stage_ready = true;
}

// scratch of the product for one precision (0 = FP64, 1 = mixed), allocated before any launch
// (and before a graph capture, which may not allocate)
static void heff_buffers(Ctx& c, Super& sb, int prec) {
  if (prec == 0) {
    c.part64.alloc(std::max<int64_t>(sb.p_elems, 1));
    c.xpad64.alloc(sb.pad_size);
    c.ygraph64.alloc(std::max<int64_t>(sb.size, 1));
    if (sb.n_big_blocks) {
      c.T.alloc(std::max<int64_t>(sb.big_t_elems, 1));
      c.bigpart64.alloc(std::max<int64_t>(sb.big_p_elems, 1));
    }
  } else {
    c.f32b.alloc(std::max<int64_t>(sb.size, 1));
    c.part32.alloc(std::max<int64_t>(sb.p_elems, 1));
    c.xpad32.alloc(sb.pad_size);
    if (sb.n_big_blocks) {
      c.f32T.alloc(std::max<int64_t>(sb.big_t_elems, 1));
      c.bigpart32.alloc(std::max<int64_t>(sb.big_p_elems, 1));
    }
  }
}

// the product's kernels after the staging of psi: small blocks, fused tiles, grouped passes
// of the big output blocks and their reductions.  FP64 writes psi' to y64; the mixed path to
// the FP32 buffer c.f32b.  Every psi' element is written by exactly one fused tile or one
// grouped-GEMM task (blocks without terms get zero-term tiles or tasks), so no clearing pass
// is needed.
static void heff_core(Ctx& c, Super& sb, int prec, double* y64, cudaStream_t st) {
  if (prec == 0) {
    HeffPtrs<double> ptr{};
    ptr.L[0] = sb.L.data.p;
    ptr.R[0] = sb.R.data.p;
    ptr.X[0] = c.xpad64.p;
    ptr.Y[0] = y64;
    ptr.P[0] = c.part64.p;
    heff_small<double>(sb.stiles.p, sb.n_stiles, sb.fitems.p, ptr, st);
    heff_fused<double>(sb.ftiles.p, sb.n_ftiles, sb.fitems.p, sb.fred.p, sb.n_fred, ptr,
                       st);
    if (sb.n_big_blocks) {
      Bases<double> bb{};
      bb.p[B_LOPS] = sb.L.data.p;
      bb.p[B_ROPS] = sb.R.data.p;
      bb.p[B_X] = c.xpad64.p;
      bb.p[B_Y] = y64;
      bb.p[B_T] = c.T.p;
      bb.p[B_Z] = c.bigpart64.p;
      run_gemm_tasks<double>(sb.big1, bb, 1, st);
      run_gemm_tasks<double>(sb.big2, bb, 1, st);
      HeffPtrs<double> rp{};
      rp.Y[0] = y64;
      rp.P[0] = c.bigpart64.p;
      heff_reduce<double>(sb.big_red.p, sb.n_big_red, rp, st);
    }
  } else {
    HeffPtrs<float> ptr{};
    ptr.L[0] = sb.L.data32.p;
    ptr.R[0] = sb.R.data32.p;
    ptr.X[0] = c.xpad32.p;
    ptr.Y[0] = c.f32b.p;
    ptr.P[0] = c.part32.p;
    heff_small<float>(sb.stiles.p, sb.n_stiles, sb.fitems.p, ptr, st);
    heff_tc(sb.ftiles.p, sb.n_ftiles, sb.fitems.p, sb.fred.p, sb.n_fred, ptr, st);
    if (sb.n_big_blocks) {
      Bases<void> bb{};
      bb.p[B_LOPS] = sb.L.data32.p;
      bb.p[B_ROPS] = sb.R.data32.p;
      bb.p[B_X] = c.xpad32.p;
      bb.p[B_Y] = c.f32b.p;
      bb.p[B_T] = c.f32T.p;
      bb.p[B_Z] = c.bigpart32.p;
      run_gemm_tasks_tc<float, float, float>(sb.big1, bb, 1, st);
      run_gemm_tasks_tc<float, float, float>(sb.big2, bb, 1, st);
      HeffPtrs<float> rp{};
      rp.Y[0] = c.f32b.p;
      rp.P[0] = c.bigpart32.p;
      heff_reduce<float>(sb.big_red.p, sb.n_big_red, rp, st);
    }
  }
}

// the scratch pointers a captured product reads and writes (a reallocation invalidates it)
static void heff_graph_key(const Ctx& c, int prec, const void* (&k)[6]) {
  if (prec == 0) {
    const void* v[6] = {c.part64.p, c.xpad64.p, c.ygraph64.p, c.T.p, c.bigpart64.p, nullptr};
    for (int i = 0; i < 6; ++i) k[i] = v[i];
  } else {
    const void* v[6] = {c.f32b.p, c.part32.p, c.xpad32.p, c.f32T.p, c.bigpart32.p, nullptr};
    for (int i = 0; i < 6; ++i) k[i] = v[i];
  }
}

// capture heff_core into the superblock's graph of this precision (on a private stream:
// capture records launches without running them, and the context stream may be the legacy
// default stream, which cannot be captured)
static void heff_capture(Ctx& c, Super& sb, int prec) {
  Super::Graph& G = sb.graph[prec];
  if (!c.cap_stream) DMRG_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  DMRG_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
  try {
    heff_core(c, sb, prec, c.ygraph64.p, c.cap_stream);
  } catch (...) {
    cudaStreamEndCapture(c.cap_stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  DMRG_CUDA(cudaStreamEndCapture(c.cap_stream, &g));
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  // the captured launches were counted by DMRG_LAUNCHED; they run at every replay instead
  g_launches.fetch_sub(int64_t(n), std::memory_order_relaxed);
  if (e == cudaSuccess && n > 0) e = cudaGraphInstantiate(&G.exec, g, 0);
  cudaGraphDestroy(g);
  DMRG_CUDA(e);
  G.n_launches = int64_t(n);
  G.empty = n == 0;   // nothing to replay: stay eager
  heff_graph_key(c, prec, G.key);
}

static void heff(Ctx& c, Super& sb, const double* x, double* y, cudaStream_t st,
                 bool graph_ok = true) {
  const int prec = c.opt.precision == DMRG_FP64 ? 0 : 1;
  const int nb = int(sb.bL.size());
  heff_buffers(c, sb, prec);
  if (prec == 0)
    pad_psi<double>(x, c.xpad64.p, sb.d_src_off.p, sb.d_pad_off.p, sb.d_pad_len.p, nb, st);
  else
    pad_psi<float>(x, c.xpad32.p, sb.d_src_off.p, sb.d_pad_off.p, sb.d_pad_len.p, nb, st);
  Super::Graph& G = sb.graph[prec];
  bool replay = false;
  if (graph_ok && c.heff_graph) {
    if (G.exec) {
      const void* k[6];
      heff_graph_key(c, prec, k);
      if (!std::equal(k, k + 6, G.key)) {   // scratch moved: capture again
        DMRG_CUDA(cudaGraphExecDestroy(G.exec));
        G.exec = nullptr;
      }
    }
    // the first product of a precision runs eagerly (kernel attributes, first-use checks);
    // from the second on the captured graph is replayed
    if (!G.exec && !G.empty && G.eager >= 1) heff_capture(c, sb, prec);
    replay = G.exec != nullptr;
  }
  if (replay) {
    DMRG_CUDA(cudaGraphLaunch(G.exec, st));
    g_launches.fetch_add(G.n_launches, std::memory_order_relaxed);
    ++G.replays;
    ++c.graph_replays;
    if (prec == 0)
      DMRG_CUDA(cudaMemcpyAsync(y, c.ygraph64.p, sizeof(double) * sb.size,
                                cudaMemcpyDeviceToDevice, st));
  } else {
    heff_core(c, sb, prec, y, st);
    ++G.eager;
  }
  if (prec == 1) to_f64(c.f32b.p, y, sb.size, st);
}

// H_eff product with its device time recorded (events resolved by resolve_heff_timing)
static void heff_timed(Ctx& c, Super& sb, const double* x, double* y) {
  if (c.ev_used + 2 > int(c.ev.size())) {
    // resolve what is pending before reusing events
    sync(c);
    for (int i = 0; i + 1 < c.ev_used; i += 2) {
      float ms = 0;
      DMRG_CUDA(cudaEventElapsedTime(&ms, c.ev[i], c.ev[i + 1]));
      c.step_heff_seconds += ms * 1e-3;
    }
    c.ev_used = 0;
    while (c.ev.size() < 256) {
      cudaEvent_t e;
      DMRG_CUDA(cudaEventCreate(&e));
      c.ev.push_back(e);
    }
  }
  DMRG_CUDA(cudaEventRecord(c.ev[c.ev_used], c.stream));
  heff(c, sb, x, y, c.stream);
  DMRG_CUDA(cudaEventRecord(c.ev[c.ev_used + 1], c.stream));
  c.ev_used += 2;
  c.heff_products += 1;
  c.heff_flops += sb.flops;
  c.heff_bytes += sb.bytes;
}

static double resolve_heff_timing(Ctx& c) {
  sync(c);
  for (int i = 0; i + 1 < c.ev_used; i += 2) {
    float ms = 0;
    DMRG_CUDA(cudaEventElapsedTime(&ms, c.ev[i], c.ev[i + 1]));
    c.step_heff_seconds += ms * 1e-3;
  }
  c.ev_used = 0;
  double s = c.step_heff_seconds;
  c.heff_seconds += s;
  c.step_heff_seconds = 0;
  return s;
}

// FP64 product regardless of the context precision (energy of the mixed path)
static void heff64(Ctx& c, Super& sb, const double* x, double* y, cudaStream_t st) {
  int keep = c.opt.precision;
  c.opt.precision = DMRG_FP64;
  try {
    heff(c, sb, x, y, st, false);   // once per step: nothing to replay
  } catch (...) {
    c.opt.precision = keep;
    throw;
  }
  c.opt.precision = keep;
}

static void ensure_diag(Ctx& c, Super& sb) {
  if (sb.diag_ready) return;
  sb.diag.alloc(std::max<int64_t>(sb.size, 1));
  heff_diag(sb.dtasks.p, sb.n_dtasks, sb.dterms.p, sb.L.data.p, sb.R.data.p, sb.diag.p, c.stream);
  sb.diag_ready = true;
}

// ---------------------------------------------------------------------------------------
// Davidson
// ---------------------------------------------------------------------------------------
__global__ void k_set_hs_diag(double* H, int ld, const double* w) {
  if (threadIdx.x == 0) {
    H[0] = w[0];
    H[1] = 0.0;
    H[ld] = 0.0;
    H[ld + 1] = w[1];
  }
}

static void ensure_ws(Ctx& c, int64_t n, int sub) {
  if (c.ws_n >= n && c.ws_sub >= sub) return;
  int64_t nn = std::max<int64_t>(n, 1);
  c.V.alloc(nn * sub);
  c.AV.alloc(nn * sub);
  c.r.alloc(nn);
  c.t.alloc(nn);
  c.x.alloc(nn);
  c.Ax.alloc(nn);
  c.x1.alloc(nn);
  c.Ax1.alloc(nn);
  c.r1.alloc(nn);
  c.small.alloc(64 * 64 * 6 + 1024);
  c.partials.alloc(64 * 300);
  std::vector<const double*> ptrs(2 * sub);
  for (int j = 0; j < sub; ++j) {
    ptrs[j] = c.V.p + j * nn;
    ptrs[sub + j] = c.AV.p + j * nn;
  }
  c.vptr.upload(ptrs, c.stream);
  c.ws_n = nn;
  c.ws_sub = sub;
}

// training pairs from the saved iterates of one Davidson run (psi = converged vector)
static void harvest(Ctx& c, Super& sb, int nhist, const double* psi) {
  cudaStream_t s = c.stream;
  const int64_t n = sb.size, ld = c.ws_n;
  double* part = c.partials.p;
  c.mlp_samples.alloc(c.mlp_cap * 5);
  const int64_t count = std::min<int64_t>(c.mlp_per_iter, n);
  if (count <= 0) return;
  const int64_t stride = std::max<int64_t>(1, n / count);
  for (int h = 0; h < nhist; ++h) {
    const double* xh = c.hist_x.p + h * ld;
    const double* rh = c.hist_r.p + h * ld;
    double* sc = c.mlp_sc.p + 16;   // {theta, |r|^2, |d|^2, x.psi, |e|^2}
    DMRG_CUDA(cudaMemcpyAsync(sc, c.hist_theta.p + h, sizeof(double), cudaMemcpyDeviceToDevice, s));
    dot(rh, rh, n, sc + 1, part, s);
    davidson_correction(rh, sb.diag.p, sc, n, c.hist_tmp.p, s);
    dot(c.hist_tmp.p, c.hist_tmp.p, n, sc + 2, part, s);
    dot(xh, psi, n, sc + 3, part, s);
    mlp_err_vec(xh, psi, sc, n, c.hist_tmp.p, s);
    dot(c.hist_tmp.p, c.hist_tmp.p, n, sc + 4, part, s);
    if (c.mlp_head + count > c.mlp_cap) c.mlp_head = 0;
    const int64_t start = (int64_t(h) * 131 + c.mlp_calls * 7) % stride;
    const int64_t cnt = std::min<int64_t>(count, (n - 1 - start) / stride + 1);
    mlp_harvest(rh, xh, psi, sb.diag.p, sc, n, start, stride, cnt,
                c.mlp_samples.p + c.mlp_head * 5, s);
    c.mlp_head += cnt;
    // filled prefix of the ring: the slots beyond the furthest write were never written
    c.mlp_nsamp = std::max<int64_t>(c.mlp_nsamp, c.mlp_head);
  }
  ++c.mlp_calls;
}

struct DavResult {
  double theta = 0, resid = 0;
  double theta1 = NAN, resid1 = 0;   // second state (two-state targeting)
  int nprod = 0;
  bool converged = false;
  double heff_seconds = 0;
};

// Davidson as a resumable run: dav_begin prepares the first vector, every H_eff product
// is requested through (px -> py), dav_after_product consumes it and either requests the
// next product or finishes.  davidson() drives one run; batch mode drives several runs
// with one fused product launch per iteration.
struct DavRun {
  Super* sb = nullptr;
  int64_t n = 0, ld = 0;
  int sub = 0, k = 0, nprod = 0, nhist = 0;
  bool use_mlp = false, done = false;
  DavResult res;
  double* out = nullptr;
  double* px = nullptr;   // pending product: py = H_eff px
  double* py = nullptr;
  int nroots = 1;                    // 2: the two lowest states
  const double* guess1 = nullptr;    // second guess, enters the subspace first
  double* out1 = nullptr;            // second state's vector
};

static const int kHist = 8;

struct DavPtrs {
  double *Hs, *w, *Y, *scr, *sc, *part;
  const double* const* Vp;
  const double* const* AVp;
  DavPtrs(Ctx& c, int sub) {
    Hs = c.small.p;              // 64 x 64, row k holds <v_i, H v_k>, i <= k
    w = Hs + 64 * 64;            // Ritz values, ascending
    Y = w + 64;                  // 64 x 64, row j = coefficients of the j-th Ritz vector
    scr = Y + 64 * 64;           // 2 x 64 x 64 scratch for the Ritz solve
    sc = scr + 2 * 64 * 64;      // device scalars
    part = c.partials.p;
    Vp = c.vptr.p;
    AVp = c.vptr.p + sub;
  }
};

static void dav_readback(Ctx& c, const double* d, int cnt, double* h) {
  if (!c.h_words) DMRG_CUDA(cudaMallocHost(&c.h_words, sizeof(double) * 64));
  DMRG_REQUIRE(cnt <= 64, DMRG_EINVAL, "internal: readback too long");
  DMRG_CUDA(cudaMemcpyAsync(c.h_words, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c.stream));
  sync(c);
  for (int i = 0; i < cnt; ++i) h[i] = c.h_words[i];
}
static void dav_d2d(Ctx& c, double* dst, const double* src, int64_t n) {
  DMRG_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.stream));
}

static void dav_begin(Ctx& c, Super& sb, const double* guess, double* out, DavRun& R,
                      const double* guess1 = nullptr, double* out1 = nullptr) {
  R = DavRun();
  R.sb = &sb;
  R.n = sb.size;
  R.nroots = out1 ? 2 : 1;
  R.guess1 = guess1;
  R.out1 = out1;
  R.sub = std::max(4, std::min(64, c.opt.dav_max_sub));
  R.out = out;
  ensure_ws(c, R.n, R.sub);
  ensure_diag(c, sb);
  R.ld = c.ws_n;
  R.use_mlp = c.opt.precond == DMRG_PRECOND_MLP && c.mlp_trained && R.nroots == 1;
  if (c.mlp_harvest) {
    c.hist_x.alloc(kHist * R.ld);
    c.hist_r.alloc(kHist * R.ld);
    c.hist_theta.alloc(kHist);
    c.hist_tmp.alloc(R.ld);
  }
  c.mlp_sc.alloc(64);
  DavPtrs P(c, R.sub);
  double* v0 = c.V.p;
  dav_d2d(c, v0, guess, R.n);
  dot(v0, v0, R.n, P.sc, P.part, c.stream);
  scale_vec(v0, R.n, P.sc, 1, c.stream);
  R.px = v0;
  R.py = c.AV.p;
}

static void dav_finish(Ctx& c, DavRun& R) {
  Super& sb = *R.sb;
  DavPtrs P(c, R.sub);
  const int64_t n = R.n;
  double h[2];
  dot(c.x.p, c.x.p, n, P.sc + 4, P.part, c.stream);
  scale_vec(c.x.p, n, P.sc + 4, 1, c.stream);
  if (c.opt.precision != DMRG_FP64) {
    // energy of the mixed path: FP64 Rayleigh quotient of the converged vector, issued on
    // the context's second stream; dav_energy() waits for it
    if (!c.rq_stream) {
      DMRG_CUDA(cudaStreamCreateWithFlags(&c.rq_stream, cudaStreamNonBlocking));
      DMRG_CUDA(cudaEventCreateWithFlags(&c.rq_in, cudaEventDisableTiming));
      DMRG_CUDA(cudaEventCreateWithFlags(&c.rq_out, cudaEventDisableTiming));
    }
    if (!c.h_words) DMRG_CUDA(cudaMallocHost(&c.h_words, sizeof(double) * 64));
    c.rq_part.alloc(64 * 300);
    c.part64.alloc(std::max<int64_t>(sb.p_elems, 1));
    c.xpad64.alloc(sb.pad_size);
    DMRG_CUDA(cudaEventRecord(c.rq_in, c.stream));   // the normalized vector is ready
    c.rq_sb = &sb;
    c.rq_n = n;
    c.rq_sc = P.sc + 5;
    c.rq_todo = true;   // launched by launch_rq (the truncation first gets the GPU)
    c.rq_pending = true;
  }
  (void)h;
  dav_d2d(c, R.out, c.x.p, n);
  if (R.nroots == 2 && R.k >= 2) {
    dot(c.x1.p, c.x1.p, n, P.sc + 8, P.part, c.stream);
    scale_vec(c.x1.p, n, P.sc + 8, 1, c.stream);
    dav_d2d(c, R.out1, c.x1.p, n);
  }
  if (c.mlp_harvest && R.nhist > 0) harvest(c, sb, R.nhist, c.x.p);
  R.done = true;
  R.px = R.py = nullptr;
}

// consume the product of vector k (py = H v_k), then either finish or request the next
static void dav_after_product(Ctx& c, DavRun& R) {
  Super& sb = *R.sb;
  cudaStream_t s = c.stream;
  DavPtrs P(c, R.sub);
  const int64_t n = R.n, ld = R.ld;
  auto vec = [&](int j) { return c.V.p + j * ld; };
  auto avec = [&](int j) { return c.AV.p + j * ld; };
  multidot(P.Vp, R.k + 1, avec(R.k), n, P.Hs + 64 * R.k, P.part, s);
  ++R.k;
  ++R.nprod;
  const double tol = c.opt.dav_tol;
  double h[4];
  // Ritz pair of the projected matrix, residual r = H x - theta x
  ritz_solve(P.Hs, 64, R.k, P.scr, P.w, P.Y, s);
  lincomb(P.Vp, P.Y, R.k, n, c.x.p, 0.0, 1.0, s);
  lincomb(P.AVp, P.Y, R.k, n, c.Ax.p, 0.0, 1.0, s);
  davidson_residual(c.x.p, c.Ax.p, P.w, n, c.r.p, s);
  dot(c.r.p, c.r.p, n, P.sc + 1, P.part, s);
  DMRG_CUDA(cudaMemcpyAsync(P.sc, P.w, sizeof(double), cudaMemcpyDeviceToDevice, s));
  // second state once the subspace holds two vectors: Ritz pair 1 and its residual
  const bool two = R.nroots == 2 && R.k >= 2;
  if (two) {
    lincomb(P.Vp, P.Y + 64, R.k, n, c.x1.p, 0.0, 1.0, s);
    lincomb(P.AVp, P.Y + 64, R.k, n, c.Ax1.p, 0.0, 1.0, s);
    davidson_residual(c.x1.p, c.Ax1.p, P.w + 1, n, c.r1.p, s);
    dot(c.r1.p, c.r1.p, n, P.sc + 3, P.part, s);   // sc[2..3] are free until the next step
    DMRG_CUDA(cudaMemcpyAsync(P.sc + 2, P.w + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  dav_readback(c, P.sc, two ? 4 : 2, h);
  const double theta = h[0], rn = std::sqrt(std::max(h[1], 0.0));
  R.res.theta = theta;
  R.res.resid = rn;
  R.res.nprod = R.nprod;
  const double rn1 = two ? std::sqrt(std::max(h[3], 0.0)) : 0.0;
  if (two) {
    R.res.theta1 = h[2];
    R.res.resid1 = rn1;
  }
  if (c.mlp_harvest && R.nhist < kHist) {   // iterate, residual and Ritz value for training
    dav_d2d(c, c.hist_x.p + R.nhist * ld, c.x.p, n);
    dav_d2d(c, c.hist_r.p + R.nhist * ld, c.r.p, n);
    DMRG_CUDA(cudaMemcpyAsync(c.hist_theta.p + R.nhist, P.w, sizeof(double),
                              cudaMemcpyDeviceToDevice, s));
    ++R.nhist;
  }
  // FP32 products cannot resolve residuals below ~1e-7 of |H|: relative floor
  const double tol_eff =
      c.opt.precision == DMRG_FP64 ? tol : std::max(tol, 1e-6 * std::max(1.0, std::fabs(theta)));
  const bool conv = rn <= tol_eff && (R.nroots == 1 || (two && rn1 <= tol_eff));
  if (conv || R.nprod >= c.opt.dav_max_iter) {
    R.res.converged = conv;
    dav_finish(c, R);
    return;
  }
  if (R.guess1 && R.k == 1) {   // the second guess enters the subspace before corrections
    dav_d2d(c, c.t.p, R.guess1, n);
    R.guess1 = nullptr;
    dot(c.t.p, c.t.p, n, P.sc + 2, P.part, s);
    for (int pass = 0; pass < 2; ++pass) {
      multidot(P.Vp, R.k, c.t.p, n, P.sc + 32, P.part, s);
      lincomb(P.Vp, P.sc + 32, R.k, n, c.t.p, 1.0, -1.0, s);
    }
    dot(c.t.p, c.t.p, n, P.sc + 3, P.part, s);
    dav_readback(c, P.sc + 2, 2, h);
    const double gn0 = std::sqrt(std::max(h[0], 0.0)), gn = std::sqrt(std::max(h[1], 0.0));
    if (gn > 1e-14 * std::max(gn0, 1e-300)) {
      dav_d2d(c, vec(R.k), c.t.p, n);
      scale_vec(vec(R.k), n, P.sc + 3, 1, s);
      R.px = vec(R.k);
      R.py = avec(R.k);
      return;
    }
  }
  // correction of the lowest state whose residual is above the tolerance:
  // t = r / (theta - D), clamped (diagonal), or the learned map
  const int j = (two && rn <= tol_eff) ? 1 : 0;
  davidson_correction(j ? c.r1.p : c.r.p, sb.diag.p, P.w + j, n, c.t.p, s);
  if (R.use_mlp) {
    double* fs = c.mlp_sc.p + 8;
    DMRG_CUDA(cudaMemcpyAsync(fs, P.w, sizeof(double), cudaMemcpyDeviceToDevice, s));
    dot(c.r.p, c.r.p, n, fs + 1, P.part, s);
    dot(c.t.p, c.t.p, n, fs + 2, P.part, s);
    c.mlp_feat.alloc(n * 4);
    mlp_features<float>(c.r.p, c.x.p, sb.diag.p, fs, n, c.mlp_feat.p, s);
    mlp_forward<float>(c.mlp_p.p, c.mlp_feat.p, n, c.mlp_acts, s);
    mlp_output_to_double<float>(c.mlp_acts.Y.p, c.t.p, n, s);
  }
  if (R.k >= R.sub) {   // thick restart from the two lowest Ritz vectors
    lincomb(P.Vp, P.Y + 64, R.k, n, c.x1.p, 0.0, 1.0, s);
    lincomb(P.AVp, P.Y + 64, R.k, n, c.Ax1.p, 0.0, 1.0, s);
    dav_d2d(c, vec(0), c.x.p, n);
    dav_d2d(c, vec(1), c.x1.p, n);
    dav_d2d(c, avec(0), c.Ax.p, n);
    dav_d2d(c, avec(1), c.Ax1.p, n);
    k_set_hs_diag<<<1, 32, 0, s>>>(P.Hs, 64, P.w);
    DMRG_LAUNCHED();
    R.k = 2;
  }
  dot(c.t.p, c.t.p, n, P.sc + 2, P.part, s);
  for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
    multidot(P.Vp, R.k, c.t.p, n, P.sc + 32, P.part, s);
    lincomb(P.Vp, P.sc + 32, R.k, n, c.t.p, 1.0, -1.0, s);
  }
  dot(c.t.p, c.t.p, n, P.sc + 3, P.part, s);
  dav_readback(c, P.sc + 2, 2, h);
  const double tn0 = std::sqrt(std::max(h[0], 0.0)), tn = std::sqrt(std::max(h[1], 0.0));
  if (tn <= 1e-14 * std::max(tn0, 1e-300)) {   // no new direction left
    dav_finish(c, R);
    return;
  }
  dav_d2d(c, vec(R.k), c.t.p, n);
  scale_vec(vec(R.k), n, P.sc + 3, 1, s);
  R.px = vec(R.k);
  R.py = avec(R.k);
}

// issue the FP64 Rayleigh quotient prepared by dav_finish (on its own stream, after the
// vector it needs); the superblock stays alive until the next truncation replaces c.prev
static void launch_rq(Ctx& c) {
  if (!c.rq_todo) return;
  c.rq_todo = false;
  DMRG_CUDA(cudaStreamWaitEvent(c.rq_stream, c.rq_in, 0));
  heff64(c, *c.rq_sb, c.x.p, c.Ax.p, c.rq_stream);
  dot(c.x.p, c.Ax.p, c.rq_n, c.rq_sc, c.rq_part.p, c.rq_stream);
  DMRG_CUDA(cudaMemcpyAsync(c.h_words + 32, c.rq_sc, sizeof(double), cudaMemcpyDeviceToHost,
                            c.rq_stream));
  DMRG_CUDA(cudaEventRecord(c.rq_out, c.rq_stream));
}

// energy of a finished run: the FP64 Rayleigh quotient of the mixed path once it is done
static void dav_energy(Ctx& c, DavResult& r) {
  launch_rq(c);
  if (!c.rq_pending) return;
  const double t0 = wall();
  DMRG_CUDA(cudaEventSynchronize(c.rq_out));
  c.t_sync += wall() - t0;
  r.theta = c.h_words[32];
  c.rq_pending = false;
}

// a Rayleigh quotient left running by the previous step of a sweep: wait, store the energy
static void settle_energy(Ctx& c) {
  if (!c.rq_target) return;
  launch_rq(c);
  const double t0 = wall();
  DMRG_CUDA(cudaEventSynchronize(c.rq_out));
  c.t_sync += wall() - t0;
  *c.rq_target = c.h_words[32];
  c.rq_target = nullptr;
  c.rq_pending = false;
}

// defer_energy: leave the Rayleigh quotient of the mixed path running (dav_energy waits)
static DavResult davidson(Ctx& c, Super& sb, const double* guess, double* out,
                          bool defer_energy = false, const double* guess1 = nullptr,
                          double* out1 = nullptr) {
  PhaseTimer tm(c.t_davidson);
  DavRun R;
  dav_begin(c, sb, guess, out, R, guess1, out1);
  while (!R.done) {
    double t0 = wall();
    heff_timed(c, sb, R.px, R.py);
    const double t1 = wall(), s0 = c.t_sync;
    dav_after_product(c, R);
    c.t_detail[16] += t1 - t0;
    c.t_detail[17] += wall() - t1 - (c.t_sync - s0);
    c.t_detail[18] += c.t_sync - s0;
    c.t_detail[19] += 1.0;
  }
  R.res.heff_seconds = resolve_heff_timing(c);
  if (!defer_energy) dav_energy(c, R.res);
  return R.res;
}


// ---------------------------------------------------------------------------------------
// truncation by the reduced density matrix and renormalization of the new block
// ---------------------------------------------------------------------------------------
struct TruncResult {
  double trunc = 0.0;
  int kept = 0;
  bool noconv = false;   // a Jacobi SVD stopped at its sweep limit (result still installed)
};

// Eigenpairs of the reduced density matrix of every sector of the truncated side (dir 0:
// enlarged left, dir 1: enlarged right) of the wave function held for the current
// superblock: eigenvalues descending into c.ew (at woff), eigenvectors as the columns of
// d x d row-major matrices into c.eVs (at roff), from the singular vectors of the
// wave-function blocks (svd.cu); sectors too large for a cluster's shared memory fall back
// to the two-sided Jacobi of the explicit density matrix (kernels.cu).  force_cluster
// (1, 8, 16) sends every sector whose shared memory fits to clusters of that size (0:
// chosen by the work of the sector).  Returns true if an SVD reached its sweep limit.
struct RdmLayout {
  int ns = 0;
  int64_t total = 0, sq = 0;
  std::vector<int64_t> roff, woff;
  std::vector<int32_t> dims;
};

static RdmLayout rdm_layout(const Layout& lay) {
  RdmLayout r;
  r.ns = lay.sec.size();
  r.roff.resize(r.ns);
  r.woff.resize(r.ns);
  r.dims.resize(r.ns);
  for (int i = 0; i < r.ns; ++i) {
    r.roff[i] = r.sq;
    r.woff[i] = r.total;
    r.dims[i] = lay.sec.d[i];
    r.sq += int64_t(lay.sec.d[i]) * lay.sec.d[i];
    r.total += lay.sec.d[i];
  }
  return r;
}

static bool rdm_eigh(Ctx& c, Super& sb, int dir, const RdmLayout& L, int force_cluster) {
  cudaStream_t s = c.stream;
  const int ns = L.ns;
  const int64_t total = L.total, sq = L.sq;
  const std::vector<int64_t>& roff = L.roff;
  const std::vector<int64_t>& woff = L.woff;
  const std::vector<int32_t>& dims = L.dims;
  // eigenpairs of rho_Q = B B^T per sector from the singular vectors of the wave-function
  // block B (svd.cu); sectors too large for a cluster's shared memory fall back to the
  // two-sided Jacobi of the explicit rho (kernels.cu)
  const bool two = c.n_roots == 2;
  const int roots = two ? 2 : 1;
  c.eVs.alloc(sq);
  c.ew.alloc(total);
  c.noconv.alloc(1);
  DMRG_CUDA(cudaMemsetAsync(c.eVs.p, 0, sizeof(double) * sq, s));
  DMRG_CUDA(cudaMemsetAsync(c.ew.p, 0, sizeof(double) * total, s));
  DMRG_CUDA(cudaMemsetAsync(c.noconv.p, 0, sizeof(int), s));
  std::vector<SvdJob> jobs[3];            // clusters of 1, 8 and 16 CTAs
  size_t smem[3] = {0, 0, 0};
  const int csize[3] = {1, 8, 16};
  std::vector<int> fallback;              // sector indices for the explicit-rho path
  for (int Q = 0; Q < ns; ++Q) {
    const int b = dir == 0 ? sb.psi_of_L[Q] : sb.psi_of_R[Q];
    if (b < 0) continue;                  // no wave-function block: rho_Q = 0
    SvdJob j;
    j.src = sb.boff[b];
    j.vs_off = roff[Q];
    j.w_off = woff[Q];
    j.D = dims[Q];
    j.e = dir == 0 ? sb.bdr[b] : sb.bdl[b];
    j.trans = dir;
    j.roots = roots;
    DMRG_REQUIRE(j.D == (dir == 0 ? sb.bdl[b] : sb.bdr[b]), DMRG_EINVAL,
                 "internal: wave-function block does not match its sector");
    const double d = j.D, E = double(j.e) * roots;
    const double cols = std::min(d, E), rows = std::max(d, E);
    const double work = cols * cols * (rows + (d < E ? d : 0.0));
    int cls = work < 4.0e5 ? 0 : (work < 8.0e6 ? 1 : 2);
    if (force_cluster) cls = force_cluster == 1 ? 0 : force_cluster == 8 ? 1 : 2;
    while (cls < 3 && svd_smem_bytes(j, csize[cls]) > svd_smem_limit()) ++cls;
    if (cls == 3) {
      fallback.push_back(Q);
      continue;
    }
    jobs[cls].push_back(j);
    smem[cls] = std::max(smem[cls], svd_smem_bytes(j, csize[cls]));
  }
  DevBuf<SvdJob> djobs[3];
  for (int k = 0; k < 3; ++k) {
    if (jobs[k].empty()) continue;
    djobs[k].upload(jobs[k], s);
    svd_jacobi(djobs[k].p, int(jobs[k].size()), csize[k], smem[k], c.psi.p,
               two ? c.psi1.p : c.psi.p, c.ew.p, c.eVs.p, c.noconv.p, s);
  }
  c.t_detail[20] += double(fallback.size());
  if (!fallback.empty()) {
    // rho = psi psi^T (or the average over the two targeted states) for these sectors
    const double wgt = two ? 0.5 : 1.0;
    TaskList R;
    std::vector<int64_t> foff, fwoff;
    std::vector<int32_t> fdim;
    for (int Q : fallback) {
      const int b = dir == 0 ? sb.psi_of_L[Q] : sb.psi_of_R[Q];
      const int dL = sb.bdl[b], dR = sb.bdr[b];
      DMRG_REQUIRE(dims[Q] <= 1024, DMRG_EINVAL, "sector dimension above 1024 not supported");
      if (dir == 0) {
        R.begin_task(Operand{roff[Q], B_Y, dL}, dL, dL);
        R.add_term(Operand{sb.boff[b], B_X, dR}, Operand{sb.boff[b], B_X, dR}, dR, 2, wgt);
        if (two)
          R.add_term(Operand{sb.boff[b], B_Z, dR}, Operand{sb.boff[b], B_Z, dR}, dR, 2, wgt);
      } else {
        R.begin_task(Operand{roff[Q], B_Y, dR}, dR, dR);
        R.add_term(Operand{sb.boff[b], B_X, dR}, Operand{sb.boff[b], B_X, dR}, dL, 1, wgt);
        if (two)
          R.add_term(Operand{sb.boff[b], B_Z, dR}, Operand{sb.boff[b], B_Z, dR}, dL, 1, wgt);
      }
      foff.push_back(roff[Q]);
      fwoff.push_back(woff[Q]);
      fdim.push_back(dims[Q]);
    }
    c.rho.alloc(sq);
    c.eV.alloc(sq);
    DMRG_CUDA(cudaMemsetAsync(c.rho.p, 0, sizeof(double) * sq, s));
    DevTaskList dR;
    {
      int64_t be[NBASE] = {0};
      be[B_X] = sb.size;
      be[B_Y] = sq;
      if (two) be[B_Z] = sb.size;
      dR.build(R, be, s);
    }
    Bases<double> bb{};
    bb.p[B_X] = c.psi.p;
    bb.p[B_Y] = c.rho.p;
    if (two) bb.p[B_Z] = c.psi1.p;
    run_gemm_tasks<double>(dR, bb, 1, s);
    DevBuf<int64_t> dfo, dfw;
    DevBuf<int32_t> dfd;
    dfo.upload(foff, s);
    dfw.upload(fwoff, s);
    dfd.upload(fdim, s);
    batched_eigh2(dfo.p, dfw.p, dfd.p, int(fallback.size()), c.rho.p, c.eV.p, c.eVs.p, c.ew.p,
                  1, 1, s);
    sync(c);   // the uploaded tables live until here
  }
  int noconv = 0;
  DMRG_CUDA(cudaMemcpyAsync(&noconv, c.noconv.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  sync(c);   // the job tables live until here
  return noconv != 0;
}

static TruncResult truncate_renormalize(Ctx& c, int p, int dir, int M) {
  wait_prefetch(c);   // a plan being made reads stored blocks; this changes one
  PhaseTimer tm(c.t_truncate);
  DMRG_REQUIRE(c.sb && c.sb->p == p && c.psi_valid && c.psi_p == p, DMRG_EINVAL,
               "no eigenvector held for this position (call dmrg_davidson first)");
  DMRG_REQUIRE(c.n_roots == 1 || c.psi1_valid, DMRG_EINVAL,
               "no second targeted state held for this position");
  DMRG_REQUIRE(dir == 0 || dir == 1, DMRG_EINVAL, "dir must be 0 or 1");
  DMRG_REQUIRE(M >= 1, DMRG_EINVAL, "M must be positive");
  Super& sb = *c.sb;
  cudaStream_t s = c.stream;
  const Layout& lay = dir == 0 ? sb.Ll : sb.Rl;
  const RdmLayout RL = rdm_layout(lay);
  const int ns = RL.ns;
  const int64_t total = RL.total;
  const std::vector<int64_t>& roff = RL.roff;
  const std::vector<int64_t>& woff = RL.woff;
  const std::vector<int32_t>& dims = RL.dims;
  // dynamic block state selection: M is the ceiling, dbss_min the floor
  const bool dbss = c.dbss_target > 0.0;
  const int floor_m = dbss ? std::min(c.dbss_min, M) : M;
  Iso iso;
  TruncResult tr;
  if (total <= floor_m) {
    launch_rq(c);
    identity_iso(c, lay, iso);
    tr.trunc = 0.0;
    tr.kept = int(total);
  } else {
    const bool noconv = rdm_eigh(c, sb, dir, RL, c.svd_cluster);
    if (noconv) {
      tr.noconv = true;
      c.eig_noconv += 1;
    }
    int64_t np2 = 1;
    while (np2 < total) np2 <<= 1;
    c.sel.alloc(np2 + 4 * int64_t(ns) + 16);
    DevBuf<int64_t> droff, dwoff, duoff;
    DevBuf<int32_t> ddim, dkept;
    droff.upload(roff, s);
    dwoff.upload(woff, s);
    ddim.upload(dims, s);
    double* lamM = c.sel.p + np2;
    double* kw = lamM + 8;
    kth_largest(c.ew.p, total, std::min<int64_t>(M, total), floor_m, dbss ? c.dbss_target : 0.0,
                c.sel.p, lamM, s);
    dkept.alloc(ns);
    count_kept(dwoff.p, ddim.p, ns, c.ew.p, lamM, dkept.p, kw, s);
    std::vector<int32_t> kept(ns);
    std::vector<double> kwh(ns);
    DMRG_CUDA(cudaMemcpyAsync(kept.data(), dkept.p, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, s));
    DMRG_CUDA(cudaMemcpyAsync(kwh.data(), kw, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    sync(c);
    launch_rq(c);   // the density-matrix decomposition is done: the energy may take the GPU
    iso.lay = lay;
    iso.m.assign(ns, 0);
    iso.uoff.assign(ns, 0);
    int64_t uo = 0;
    double kept_w = 0.0;
    for (int i = 0; i < ns; ++i) {
      iso.m[i] = kept[i];
      iso.uoff[i] = uo;
      uo += int64_t(dims[i]) * kept[i];
      tr.kept += kept[i];
      kept_w += kwh[i];
    }
    tr.trunc = std::max(0.0, 1.0 - kept_w);
    iso.data.alloc(std::max<int64_t>(uo, 1));
    duoff.upload(iso.uoff, s);
    gather_u(droff.p, ddim.p, dkept.p, duoff.p, ns, c.eVs.p, iso.data.p, s);
    sync(c);
    iso.identity = false;
  }
  finish_iso_index(iso);
  Blk& dst = dir == 0 ? c.left[p] : c.right[p];
  dst.valid = false;
  OpSet ops;
  project(c, dir == 0 ? sb.L : sb.R, iso, ops);
  dst.ops = std::move(ops);
  dst.iso = std::move(iso);
  dst.valid = true;
  dst.gen = ++g_blk_gen;
  if (c.rq_pending && c.rq_sb != c.sb.get()) {   // a Rayleigh quotient still reads c.prev
    launch_rq(c);
    DMRG_CUDA(cudaEventSynchronize(c.rq_out));
  }
  c.prev = std::move(c.sb);   // layouts of the superblock psi belongs to
  return tr;
}

// ---------------------------------------------------------------------------------------
// prediction of the next wave function (White's transformation)
// ---------------------------------------------------------------------------------------
static void uniform_guess(Ctx& c, Super& sb, double* g) {
  fill_value(g, sb.size, 1.0 / std::sqrt(double(std::max<int64_t>(sb.size, 1))), c.stream);
}

// src: a vector of the previous step (its ground state by default)
static void predict(Ctx& c, Super& sb, int p, int dir, double* g, const double* src = nullptr) {
  PhaseTimer tm(c.t_predict);
  cudaStream_t s = c.stream;
  if (!src) src = c.psi.p;
  if (!c.psi_valid || !c.prev) {
    uniform_guess(c, sb, g);
    return;
  }
  Super& pr = *c.prev;
  if (pr.p == p) {
    DMRG_REQUIRE(pr.size == sb.size, DMRG_EINVAL, "internal: layout changed at turn");
    DMRG_CUDA(cudaMemcpyAsync(g, src, sizeof(double) * sb.size, cudaMemcpyDeviceToDevice, s));
    return;
  }
  TaskList A, B;
  int64_t xoff = 0;
  int64_t bu_n = 0, bv_n = 0;
  Bases<double> bb{};
  if (dir == 0 && pr.p == p - 1) {
    const Iso& U = c.left[p - 1].iso;     // new left block of bond p-1
    const Iso& Ur = c.right[p].iso;       // right block of bond p: (site p+1) x (right of p+1)
    const SectorSet& lsec = c.left[p - 1].ops.sec;
    const SectorSet& rsec = c.right[p].ops.sec;
    DMRG_REQUIRE(Ur.lay.sec.q == sb.Rl.sec.q && Ur.lay.sec.d == sb.Rl.sec.d, DMRG_EINVAL,
                 "internal: right basis does not refer to the current enlarged space");
    for (size_t b = 0; b < pr.bL.size(); ++b) {
      const int QLo = pr.bL[b], QRo = pr.bR[b], dL = pr.bdl[b], dR = pr.bdr[b];
      const int newl = U.kept_idx[QLo];
      if (newl < 0) continue;
      const int m = U.m[QLo];
      A.begin_task(Operand{xoff, B_T, dR}, m, dR);
      A.add_term(Operand{U.uoff[QLo], B_U, m}, Operand{pr.boff[b], B_X, dR}, dL, 1, 1.0);
      for (int sg = 0; sg < 2; ++sg) {
        const int rb = pr.Rl.pblk[QRo][sg];
        if (rb < 0) continue;
        const int coff = pr.Rl.poff[QRo][sg], dr = rsec.d[rb];
        const int er = Ur.enl_idx[rb];
        QN qn = sg ? lsec.q[newl] + c.chain.q[p] : lsec.q[newl];
        const int QLn = sb.Ll.sec.find(qn);
        if (QLn < 0 || sb.Ll.pblk[QLn][sg] != newl) continue;
        const int bn = sb.psi_of_L[QLn];
        if (bn < 0 || sb.bR[bn] != er) continue;
        const int rof = sb.Ll.poff[QLn][sg], dRn = sb.bdr[bn];
        B.begin_task(Operand{sb.boff[bn] + int64_t(rof) * dRn, B_Y, dRn}, m, dRn);
        B.add_term(Operand{xoff + coff, B_T, dR}, Operand{Ur.uoff[er], B_V, dr}, dr, 2, 1.0);
      }
      xoff += int64_t(m) * dR;
    }
    bb.p[B_U] = U.data.p;
    bb.p[B_V] = Ur.data.p;
    bu_n = U.data.n;
    bv_n = Ur.data.n;
  } else if (dir == 1 && pr.p == p + 1) {
    const Iso& V = c.right[p + 1].iso;    // new right block of bond p+1
    const Iso& Ul = c.left[p].iso;        // left block of bond p: (left of p-1) x (site p)
    const SectorSet& rsec = c.right[p + 1].ops.sec;
    const SectorSet& lsec = c.left[p].ops.sec;
    DMRG_REQUIRE(Ul.lay.sec.q == sb.Ll.sec.q && Ul.lay.sec.d == sb.Ll.sec.d, DMRG_EINVAL,
                 "internal: left basis does not refer to the current enlarged space");
    for (size_t b = 0; b < pr.bL.size(); ++b) {
      const int QLo = pr.bL[b], QRo = pr.bR[b], dL = pr.bdl[b], dR = pr.bdr[b];
      const int newr = V.kept_idx[QRo];
      if (newr < 0) continue;
      const int m = V.m[QRo];
      A.begin_task(Operand{xoff, B_T, m}, dL, m);
      A.add_term(Operand{pr.boff[b], B_X, dR}, Operand{V.uoff[QRo], B_U, m}, dR, 0, 1.0);
      for (int sg = 0; sg < 2; ++sg) {
        const int lb = pr.Ll.pblk[QLo][sg];
        if (lb < 0) continue;
        const int roff = pr.Ll.poff[QLo][sg], dl = lsec.d[lb];
        const int el = Ul.enl_idx[lb];
        QN qn = sg ? rsec.q[newr] + c.chain.q[p + 1] : rsec.q[newr];
        const int QRn = sb.Rl.sec.find(qn);
        if (QRn < 0 || sb.Rl.pblk[QRn][sg] != newr) continue;
        const int bn = sb.psi_of_L[el];
        if (bn < 0 || sb.bR[bn] != QRn) continue;
        const int cof = sb.Rl.poff[QRn][sg], dRn = sb.bdr[bn];
        B.begin_task(Operand{sb.boff[bn] + cof, B_Y, dRn}, sb.bdl[bn], m);
        B.add_term(Operand{Ul.uoff[el], B_V, dl}, Operand{xoff + int64_t(roff) * m, B_T, m}, dl,
                   0, 1.0);
      }
      xoff += int64_t(dL) * m;
    }
    bb.p[B_U] = V.data.p;
    bb.p[B_V] = Ul.data.p;
    bu_n = V.data.n;
    bv_n = Ul.data.n;
  } else {
    uniform_guess(c, sb, g);
    return;
  }
  c.tmp.alloc(std::max<int64_t>(xoff, 1));
  DMRG_CUDA(cudaMemsetAsync(g, 0, sizeof(double) * sb.size, s));
  DevTaskList dA, dB;
  {
    int64_t be[NBASE] = {0};
    be[B_X] = pr.size;
    be[B_T] = c.tmp.n;
    be[B_Y] = sb.size;
    be[B_U] = bu_n;
    be[B_V] = bv_n;
    dA.build(A, be, s);
    dB.build(B, be, s);
  }
  bb.p[B_X] = const_cast<double*>(src);   // read only
  bb.p[B_T] = c.tmp.p;
  bb.p[B_Y] = g;
  run_gemm_tasks<double>(dA, bb, 1, s);
  run_gemm_tasks<double>(dB, bb, 1, s);
  c.small.alloc(64 * 64 * 6 + 1024);
  c.partials.alloc(64 * 300);
  double* sc = c.small.p + 64 * 64 * 6;
  dot(g, g, sb.size, sc, c.partials.p, s);
  double nrm2 = 0;
  dav_readback(c, sc, 1, &nrm2);
  if (!(nrm2 > 0.0)) {
    uniform_guess(c, sb, g);
    return;
  }
  scale_vec(g, sb.size, sc, 1, s);
}

// ---------------------------------------------------------------------------------------
// blocks from the starting state
// ---------------------------------------------------------------------------------------
static void build_blocks(Ctx& c, const dmrg_mps_init* init) {
  wait_prefetch(c);
  if (c.pf.st) DMRG_CUDA(cudaStreamSynchronize(c.pf.st));
  c.pf.active = false;
  c.pf.dev_ready = false;
  c.pf.out = OpSet();
  const int N = c.N;
  cudaStream_t s = c.stream;
  c.left.clear();
  c.right.clear();
  c.left.resize(N);
  c.right.resize(N);
  c.sb.reset();
  c.prev.reset();
  c.psi_valid = false;
  c.built = false;
  {
    OpSet vac = vacuum_ops(int(c.mpo.labels[0].size()), 0, s);
    Layout lay;
    OpSet E;
    enlarge(c, vac, 0, true, lay, E);
    identity_iso(c, lay, c.left[0].iso);
    project(c, E, c.left[0].iso, c.left[0].ops);
    c.left[0].valid = true;
    c.left[0].gen = ++g_blk_gen;
  }
  {
    OpSet vac = vacuum_ops(int(c.mpo.labels[N].size()), 0, s);
    Layout lay;
    OpSet E;
    enlarge(c, vac, N - 1, false, lay, E);
    identity_iso(c, lay, c.right[N - 2].iso);
    project(c, E, c.right[N - 2].iso, c.right[N - 2].ops);
    c.right[N - 2].valid = true;
    c.right[N - 2].gen = ++g_blk_gen;
  }
  DMRG_REQUIRE(init != nullptr, DMRG_EINVAL, "starting state is NULL");
  DMRG_REQUIRE(init->n_bonds == N - 4, DMRG_EINVAL, "starting state must cover bonds N-3..2");
  for (int bi = 0; bi < init->n_bonds; ++bi) {
    const int b = init->bonds[bi];
    DMRG_REQUIRE(b == N - 3 - bi, DMRG_EINVAL, "starting state bonds must be N-3, N-4, ..., 2");
    Layout lay;
    OpSet E;
    enlarge(c, c.right[b + 1].ops, b + 1, false, lay, E);
    Iso iso;
    iso.lay = lay;
    const int ns = lay.sec.size();
    iso.m.assign(ns, 0);
    iso.uoff.assign(ns, 0);
    std::vector<int64_t> src(ns, -1);
    for (int x = init->bond_ptr[bi]; x < init->bond_ptr[bi + 1]; ++x) {
      const int32_t* r = init->sec + 5 * int64_t(x);
      QN q{r[0], r[1], r[2]};
      const int idx = lay.sec.find(q);
      DMRG_REQUIRE(idx >= 0 && lay.sec.d[idx] == r[3] && r[4] >= 0 && r[4] <= r[3], DMRG_EINVAL,
                   "starting state does not match the sector structure at bond " +
                       std::to_string(b));
      DMRG_REQUIRE(init->u_off[x + 1] - init->u_off[x] == int64_t(r[3]) * r[4], DMRG_EINVAL,
                   "starting state isometry size mismatch");
      iso.m[idx] = r[4];
      src[idx] = init->u_off[x];
    }
    int64_t uo = 0;
    for (int i = 0; i < ns; ++i) {
      iso.uoff[i] = uo;
      uo += int64_t(lay.sec.d[i]) * iso.m[i];
    }
    std::vector<double> h(std::max<int64_t>(uo, 1), 0.0);
    for (int i = 0; i < ns; ++i)
      if (iso.m[i] > 0)
        std::memcpy(h.data() + iso.uoff[i], init->u + src[i],
                    sizeof(double) * size_t(lay.sec.d[i]) * iso.m[i]);
    iso.data.upload(h, s);
    finish_iso_index(iso);
    OpSet ops;
    project(c, E, iso, ops);
    c.right[b].ops = std::move(ops);
    c.right[b].iso = std::move(iso);
    c.right[b].valid = true;
    c.right[b].gen = ++g_blk_gen;
  }
  c.built = true;
}

// ---------------------------------------------------------------------------------------
// one two-site step
// ---------------------------------------------------------------------------------------
static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// late_energy: in a sweep, the mixed path's energy of this step is stored there once the next
// step has built its superblock (its Rayleigh quotient overlaps that host work)
// ---------------------------------------------------------------------------------------
// all-pairs orbital mutual information along a left-to-right half sweep.  The occupation
// n_i and the creation operator c+_i of every orbital i of the left block are carried
// through the renormalizations (label 2i: n_i, 2i+1: c+_i with the Jordan-Wigner string of
// the block's earlier orbitals).  At step p the pairs (i, p), i < p, are read off the
// wave function's density matrix on the enlarged left block, rho = psi psi^T per block:
//   <n_i> = sum_sigma n_i . rho[sigma sigma],  <n_i n_p> = n_i . rho[1 1],
//   <c+_i c_p> = (-1)^{N(q)} c+_i . rho[0 1]   (same species and 2m only; q: the block
//   sector of the occupied piece),
// and at the last step (p = N-3) the pairs with the right dot N-2 and with the right
// block's single orbital N-1 from the wave function's columns, whose occupations are
// explicit there: column-restricted density matrices for the diagonal terms, transition
// matrices between blocks for the hops.  Each pair's two-orbital density matrix (basis
// |n_i n_j>, off-diagonal <c+_i c_j>) then gives s_i, s_j, s_ij and I_ij = s_i + s_j - s_ij.
// ---------------------------------------------------------------------------------------
struct MiRun {
  OpSet ops;                    // carried operators on the left block of the current step
  int N = 0;
  std::vector<double> I, s;     // chain positions
};

static bool mi_piece(const Layout& L, int Q, int sg, int* off, int* len) {
  if (L.pblk[Q][sg] < 0) return false;
  const int D = L.sec.d[Q];
  *off = L.poff[Q][sg];
  *len = (sg == 0 && L.pblk[Q][1] >= 0 ? L.poff[Q][1] : D) - *off;
  return *len > 0;
}

static double mi_vn(std::initializer_list<double> w) {
  double s = 0.0;
  for (double x : w)
    if (x > 0.0) s -= x * std::log(x);
  return s;
}

// s_i, s_j and I_ij of two orbitals from <n_i>, <n_j>, <n_i n_j> and <c+_i c_j>
static void mi_pair(double ni, double nj, double nij, double h, double* si, double* sj,
                    double* I) {
  const double p11 = nij, p10 = ni - nij, p01 = nj - nij, p00 = 1.0 - ni - nj + nij;
  const double mid = 0.5 * (p01 + p10);
  const double rad = std::sqrt(0.25 * (p01 - p10) * (p01 - p10) + h * h);
  *si = mi_vn({1.0 - ni, ni});
  *sj = mi_vn({1.0 - nj, nj});
  *I = *si + *sj - mi_vn({p00, p11, mid + rad, mid - rad});
}

// the left block of bond 0 (orbital 0 alone): n_0 and c+_0 on its sectors of one state
static void mi_init(Ctx& c, MiRun& mr) {
  const OpSet& L0 = c.left[0].ops;
  DMRG_REQUIRE(c.left[0].valid, DMRG_EINVAL, "blocks are not built");
  OpSet& o = mr.ops;
  o = OpSet();
  o.sec = L0.sec;
  o.nlab = 2;
  o.lab_ptr.assign(3, 0);
  const QN q0 = c.chain.q[0], vac{0, 0, 0};
  std::vector<double> h;
  for (int s = 0; s < o.sec.size(); ++s) {
    DMRG_REQUIRE(o.sec.d[s] == 1, DMRG_EINVAL, "internal: the block of bond 0 is not one orbital");
    o.blocks.push_back(OpBlock{s, s, int64_t(h.size())});
    h.push_back(o.sec.q[s] == q0 ? 1.0 : 0.0);
  }
  o.lab_ptr[1] = int64_t(o.blocks.size());
  const int se = o.sec.find(vac), so = o.sec.find(q0);
  if (se >= 0 && so >= 0) {
    o.blocks.push_back(OpBlock{so, se, int64_t(h.size())});
    h.push_back(1.0);
  }
  o.lab_ptr[2] = int64_t(o.blocks.size());
  o.n_elems = int64_t(h.size());
  o.data.upload(h, c.stream);
  o.index_by_in();
}

// rectangle checks against the buffers they read
static void mi_check(const RectDot& t, int64_t nA, int64_t nB) {
  DMRG_REQUIRE(t.nr >= 0 && t.nc >= 0 && t.b >= 0 && t.nc <= t.ldb, DMRG_EINVAL,
               "internal: density rectangle malformed");
  if (t.nr == 0 || t.nc == 0) return;
  DMRG_REQUIRE(t.b + int64_t(t.nr - 1) * t.ldb + t.nc <= nB, DMRG_EINVAL,
               "internal: density rectangle outside its matrix");
  if (t.lda < 0) {
    DMRG_REQUIRE(t.nr == t.nc, DMRG_EINVAL, "internal: trace of a non-square rectangle");
  } else {
    DMRG_REQUIRE(t.a >= 0 && t.nc <= t.lda && t.a + int64_t(t.nr - 1) * t.lda + t.nc <= nA,
                 DMRG_EINVAL, "internal: operator rectangle outside the carried operators");
  }
}

static void mi_measure(Ctx& c, MiRun& mr, Super& sb, int p) {
  const int N = c.N;
  const bool last = p == N - 3;
  const Layout& Ll = sb.Ll;
  const Layout& Rl = sb.Rl;
  const OpSet& B = mr.ops;
  const int nsB = B.sec.size();
  DMRG_REQUIRE(c.left[p - 1].ops.sec.q == B.sec.q && c.left[p - 1].ops.sec.d == B.sec.d,
               DMRG_EINVAL, "internal: carried operators do not match the left block");
  const int nb = int(sb.bL.size());
  const QN vac{0, 0, 0};
  const QN qp = c.chain.q[p];
  auto parity = [](const QN& q) { return ((q.a + q.b) & 1) ? -1.0 : 1.0; };
  // ---- density and transition matrices of the wave function (FP64 GEMM tasks)
  TaskList T;
  int64_t roff = 0;
  auto matrix = [&](int rows, int cols) {
    const int64_t o = roff;
    T.begin_task(Operand{o, B_Y, cols}, rows, cols);
    roff += int64_t(rows) * cols;
    return o;
  };
  std::vector<int64_t> rho(nb);
  for (int b = 0; b < nb; ++b) {
    const int D = sb.bdl[b], dR = sb.bdr[b];
    rho[b] = matrix(D, D);
    T.add_term(Operand{sb.boff[b], B_X, dR}, Operand{sb.boff[b], B_X, dR}, dR, 2, 1.0);
  }
  // last step: columns of every block with the occupations of N-2 (right dot) and N-1
  struct Col {
    int off, sg, occ;
  };
  std::vector<std::vector<Col>> cols(nb);
  std::vector<int64_t> s_rd(nb, -1), s_rs(nb, -1), s_rr(nb, -1), t_rr(nb, -1);
  std::vector<int64_t> t_j[2] = {std::vector<int64_t>(nb, -1), std::vector<int64_t>(nb, -1)};
  std::vector<int> b2_j[2] = {std::vector<int>(nb, -1), std::vector<int>(nb, -1)};
  const QN q_rd = last ? c.chain.q[N - 2] : vac, q_rs = last ? c.chain.q[N - 1] : vac;
  if (last) {
    for (int b = 0; b < nb; ++b) {
      const int jR = sb.bR[b];
      const QN QR = Rl.sec.q[jR];
      for (int sg = 0; sg < 2; ++sg) {
        int off, len;
        if (!mi_piece(Rl, jR, sg, &off, &len)) continue;
        const QN r = sg ? QR - q_rd : QR;
        DMRG_REQUIRE(len == 1 && (r == vac || r == q_rs), DMRG_EINVAL,
                     "internal: the last right block is not one orbital");
        cols[b].push_back(Col{off, sg, r == q_rs ? 1 : 0});
      }
    }
    auto select = [&](int b, int want_rd, int want_rs) -> int64_t {
      std::vector<int> pick;
      for (const Col& k : cols[b])
        if ((want_rd < 0 || k.sg == want_rd) && (want_rs < 0 || k.occ == want_rs)) pick.push_back(k.off);
      if (pick.empty()) return -1;
      const int D = sb.bdl[b], dR = sb.bdr[b];
      const int64_t o = matrix(D, D);
      for (int co : pick)
        T.add_term(Operand{sb.boff[b] + co, B_X, dR}, Operand{sb.boff[b] + co, B_X, dR}, 1, 2, 1.0);
      return o;
    };
    for (int b = 0; b < nb; ++b) {
      s_rd[b] = select(b, 1, -1);
      s_rs[b] = select(b, -1, 1);
      s_rr[b] = select(b, 1, 1);
    }
    // transitions <bra| ... a_j |ket>: ket columns with orbital j occupied, bra columns of the
    // block whose left sector gained q_j with j empty and the other occupation unchanged
    const QN qj[2] = {q_rd, q_rs};
    for (int j = 0; j < 2; ++j) {
      bool need = c.chain.q[p] == qj[j];
      for (int i = 0; i < p && !need; ++i) need = c.chain.q[i] == qj[j];
      if (!need) continue;
      for (int b = 0; b < nb; ++b) {
        const int Q2 = Ll.sec.find(Ll.sec.q[sb.bL[b]] + qj[j]);
        if (Q2 < 0) continue;
        const int b2 = sb.psi_of_L[Q2];
        if (b2 < 0) continue;
        DMRG_REQUIRE(Rl.sec.q[sb.bR[b2]] == Rl.sec.q[sb.bR[b]] - qj[j], DMRG_EINVAL,
                     "internal: transition block does not conserve the target");
        std::vector<std::array<int, 3>> pairs;   // bra column, ket column, sign
        for (const Col& k : cols[b]) {
          if ((j == 0 ? k.sg : k.occ) != 1) continue;
          for (const Col& k2 : cols[b2]) {
            const bool match = j == 0 ? (k2.sg == 0 && k2.occ == k.occ) : (k2.sg == k.sg && k2.occ == 0);
            if (match) pairs.push_back({k2.off, k.off, (j == 1 && k.sg == 1) ? -1 : 1});
          }
        }
        if (pairs.empty()) continue;
        const int D = sb.bdl[b], D2 = sb.bdl[b2], dR = sb.bdr[b], dR2 = sb.bdr[b2];
        t_j[j][b] = matrix(D2, D);
        b2_j[j][b] = b2;
        for (auto& pr : pairs)
          T.add_term(Operand{sb.boff[b2] + pr[0], B_X, dR2}, Operand{sb.boff[b] + pr[1], B_X, dR},
                     1, 2, double(pr[2]));
      }
    }
    if (q_rd == q_rs) {   // hop between the right dot and the last orbital, inside a block
      for (int b = 0; b < nb; ++b) {
        int ket = -1, bra = -1;
        for (const Col& k : cols[b]) {
          if (k.sg == 0 && k.occ == 1) ket = k.off;
          if (k.sg == 1 && k.occ == 0) bra = k.off;
        }
        if (ket < 0 || bra < 0) continue;
        const int D = sb.bdl[b], dR = sb.bdr[b];
        t_rr[b] = matrix(D, D);
        T.add_term(Operand{sb.boff[b] + bra, B_X, dR}, Operand{sb.boff[b] + ket, B_X, dR}, 1, 2,
                   1.0);
      }
    }
  }
  // ---- rectangle dot products, grouped by slot
  std::vector<std::vector<RectDot>> slots;
  auto slot = [&]() {
    slots.emplace_back();
    return int(slots.size()) - 1;
  };
  auto trace = [&](int k, int64_t base, int D, int off_r, int off_c, int n, double sign) {
    slots[k].push_back(RectDot{0, base + int64_t(off_r) * D + off_c, -1, D, n, n, sign});
  };
  // n_i (x) rows/cols sigma of a D x D matrix at base, summed over both pieces (sg < 0) or
  // one piece
  auto n_dot = [&](int k, int i, int b, int64_t base, int sg_only) {
    const int Q = sb.bL[b], D = sb.bdl[b];
    for (int sg = 0; sg < 2; ++sg) {
      if (sg_only >= 0 && sg != sg_only) continue;
      int off, len;
      if (!mi_piece(Ll, Q, sg, &off, &len)) continue;
      const int s_in = Ll.pblk[Q][sg];
      const int x = B.by_in[size_t(2 * i) * nsB + s_in];
      if (x < 0) continue;
      DMRG_REQUIRE(B.sec.d[s_in] == len && B.blocks[x].so == s_in, DMRG_EINVAL,
                   "internal: occupation block does not fit its piece");
      slots[k].push_back(RectDot{B.blocks[x].off, base + int64_t(off) * D + off, len, D, len, len, 1.0});
    }
  };
  const int k_np = slot();
  std::vector<int> k_n(p), k_nn(p), k_h(p, -1);
  for (int i = 0; i < p; ++i) {
    k_n[i] = slot();
    k_nn[i] = slot();
    if (c.chain.q[i] == qp) k_h[i] = slot();
  }
  for (int b = 0; b < nb; ++b) {
    const int Q = sb.bL[b], D = sb.bdl[b];
    int o0, l0, o1, l1;
    const bool has0 = mi_piece(Ll, Q, 0, &o0, &l0), has1 = mi_piece(Ll, Q, 1, &o1, &l1);
    if (has1) trace(k_np, rho[b], D, o1, o1, l1, 1.0);
    for (int i = 0; i < p; ++i) {
      n_dot(k_n[i], i, b, rho[b], -1);
      n_dot(k_nn[i], i, b, rho[b], 1);
      if (k_h[i] >= 0 && has0 && has1) {
        const int s1 = Ll.pblk[Q][1], s0 = Ll.pblk[Q][0];
        const int x = B.by_in[size_t(2 * i + 1) * nsB + s1];
        if (x < 0) continue;
        DMRG_REQUIRE(B.blocks[x].so == s0 && B.sec.d[s0] == l0 && B.sec.d[s1] == l1, DMRG_EINVAL,
                     "internal: creation block does not fit its pieces");
        slots[k_h[i]].push_back(RectDot{B.blocks[x].off, rho[b] + int64_t(o0) * D + o1, l1, D, l0,
                                        l1, parity(B.sec.q[s1])});
      }
    }
  }
  // last step: pairs with the right dot (j = 0) and the last orbital (j = 1)
  int k_nj[2] = {-1, -1}, k_njj = -1, k_hjj = -1, k_pnj[2] = {-1, -1}, k_phj[2] = {-1, -1};
  std::vector<int> k_inj[2], k_ihj[2];
  if (last) {
    const std::vector<int64_t>* sel[2] = {&s_rd, &s_rs};
    const QN qj[2] = {q_rd, q_rs};
    k_njj = slot();
    if (q_rd == q_rs) k_hjj = slot();
    for (int j = 0; j < 2; ++j) {
      k_nj[j] = slot();
      k_pnj[j] = slot();
      if (qp == qj[j]) k_phj[j] = slot();
      k_inj[j].assign(p, -1);
      k_ihj[j].assign(p, -1);
      for (int i = 0; i < p; ++i) {
        k_inj[j][i] = slot();
        if (c.chain.q[i] == qj[j]) k_ihj[j][i] = slot();
      }
    }
    for (int b = 0; b < nb; ++b) {
      const int Q = sb.bL[b], D = sb.bdl[b];
      if (s_rr[b] >= 0) trace(k_njj, s_rr[b], D, 0, 0, D, 1.0);
      if (t_rr[b] >= 0) trace(k_hjj, t_rr[b], D, 0, 0, D, 1.0);
      for (int j = 0; j < 2; ++j) {
        const int64_t S = (*sel[j])[b];
        if (S >= 0) {
          trace(k_nj[j], S, D, 0, 0, D, 1.0);
          int o1, l1;
          if (mi_piece(Ll, Q, 1, &o1, &l1)) trace(k_pnj[j], S, D, o1, o1, l1, 1.0);
          for (int i = 0; i < p; ++i) n_dot(k_inj[j][i], i, b, S, -1);
        }
        const int64_t Tt = t_j[j][b];
        if (Tt < 0) continue;
        const int b2 = b2_j[j][b], Q2 = sb.bL[b2];
        // c+_p c_j: the left dot empty in the ket, occupied in the bra, block state unchanged
        int o0, l0, o1b, l1b;
        if (k_phj[j] >= 0 && mi_piece(Ll, Q, 0, &o0, &l0) && mi_piece(Ll, Q2, 1, &o1b, &l1b)) {
          DMRG_REQUIRE(Ll.pblk[Q][0] == Ll.pblk[Q2][1] && l0 == l1b, DMRG_EINVAL,
                       "internal: left-dot transition pieces differ");
          trace(k_phj[j], Tt, D, o1b, o0, l0, 1.0);
        }
        // c+_i c_j, i in the block: the piece of the left dot unchanged
        for (int i = 0; i < p; ++i) {
          if (k_ihj[j][i] < 0) continue;
          for (int sg = 0; sg < 2; ++sg) {
            int oi, li, oo, lo;
            if (!mi_piece(Ll, Q, sg, &oi, &li) || !mi_piece(Ll, Q2, sg, &oo, &lo)) continue;
            const int s_in = Ll.pblk[Q][sg], s_out = Ll.pblk[Q2][sg];
            const int x = B.by_in[size_t(2 * i + 1) * nsB + s_in];
            if (x < 0) continue;
            DMRG_REQUIRE(B.blocks[x].so == s_out && B.sec.d[s_in] == li && B.sec.d[s_out] == lo,
                         DMRG_EINVAL, "internal: creation block does not fit its pieces");
            const double sign = parity(B.sec.q[s_in]) * (sg ? -1.0 : 1.0);
            slots[k_ihj[j][i]].push_back(
                RectDot{B.blocks[x].off, Tt + int64_t(oo) * D + oi, li, D, lo, li, sign});
          }
        }
      }
    }
  }
  // ---- device work: the matrices, the rectangles, the sums per slot
  int64_t be[NBASE] = {0};
  be[B_X] = sb.size;
  be[B_Y] = std::max<int64_t>(roff, 1);
  DevTaskList L;
  L.build(T, be, c.stream);
  DevBuf<double> R;
  R.alloc(std::max<int64_t>(roff, 1));
  Bases<double> bb{};
  bb.p[B_X] = c.psi.p;
  bb.p[B_Y] = R.p;
  run_gemm_tasks<double>(L, bb, 1, c.stream);
  std::vector<RectDot> flat;
  std::vector<int64_t> ptr(1, 0);
  for (auto& v : slots) {
    for (const RectDot& t : v) mi_check(t, B.n_elems, roff);
    flat.insert(flat.end(), v.begin(), v.end());
    ptr.push_back(int64_t(flat.size()));
  }
  const int64_t ns = int64_t(slots.size());
  DevBuf<RectDot> dt;
  DevBuf<int64_t> dp;
  DevBuf<double> part, out;
  dt.upload(flat, c.stream);
  dp.upload(ptr, c.stream);
  part.alloc(std::max<int64_t>(int64_t(flat.size()), 1));
  out.alloc(std::max<int64_t>(ns, 1));
  rect_dots(dt.p, int64_t(flat.size()), B.data.p, R.p, part.p, c.stream);
  slot_sums(dp.p, ns, part.p, out.p, c.stream);
  std::vector<double> h(size_t(std::max<int64_t>(ns, 1)));
  DMRG_CUDA(cudaMemcpyAsync(h.data(), out.p, sizeof(double) * ns, cudaMemcpyDeviceToHost,
                            c.stream));
  sync(c);
  // ---- two-orbital density matrices of this step's pairs
  auto val = [&](int k) { return k >= 0 ? h[k] : 0.0; };
  auto put = [&](int i, int j, double ni, double nj, double nij, double hij) {
    double si, sj, I;
    mi_pair(ni, nj, nij, hij, &si, &sj, &I);
    mr.I[size_t(i) * N + j] = mr.I[size_t(j) * N + i] = I;
    if (last) {
      mr.s[i] = si;
      mr.s[j] = sj;
    }
  };
  const double np_ = h[k_np];
  for (int i = 0; i < p; ++i) put(i, p, h[k_n[i]], np_, h[k_nn[i]], val(k_h[i]));
  if (last) {
    const int jpos[2] = {N - 2, N - 1};
    for (int j = 0; j < 2; ++j) {
      const double nj = h[k_nj[j]];
      for (int i = 0; i < p; ++i) put(i, jpos[j], h[k_n[i]], nj, h[k_inj[j][i]], val(k_ihj[j][i]));
      put(p, jpos[j], np_, nj, h[k_pnj[j]], val(k_phj[j]));
    }
    put(N - 2, N - 1, h[k_nj[0]], h[k_nj[1]], h[k_njj], val(k_hjj));
  }
}

// after the truncation at p: the carried operators and those of orbital p, embedded in the
// enlarged left space (block operator (x) 1 of the site; n_p and c+_p = parity of the block
// (x) c+ of the site), renormalized with the new block's basis
static void mi_carry(Ctx& c, MiRun& mr, Super& sb, int p) {
  const Layout& Ll = sb.Ll;
  const OpSet& B = mr.ops;
  const int nsB = B.sec.size();
  const Iso& iso = c.left[p].iso;
  DMRG_REQUIRE(iso.lay.sec.q == Ll.sec.q && iso.lay.sec.d == Ll.sec.d, DMRG_EINVAL,
               "internal: the new basis does not refer to the enlarged space");
  OpSet E;
  E.sec = Ll.sec;
  E.nlab = 2 * (p + 1);
  E.lab_ptr.assign(size_t(E.nlab) + 1, 0);
  std::vector<EmbedTask> emb;
  int64_t eoff = 0;
  const int nE = Ll.sec.size();
  for (int lab = 0; lab < E.nlab; ++lab) {
    E.lab_ptr[lab] = int64_t(E.blocks.size());
    const int i = lab / 2;
    const bool cre = lab & 1;
    for (int Q = 0; Q < nE; ++Q) {
      const int Q2 = cre ? Ll.sec.find(Ll.sec.q[Q] + c.chain.q[i]) : Q;
      if (Q2 < 0) continue;
      const int Din = Ll.sec.d[Q], Dout = Ll.sec.d[Q2];
      std::vector<EmbedTask> here;
      if (i < p) {
        for (int sg = 0; sg < 2; ++sg) {
          int oi, li, oo, lo;
          if (!mi_piece(Ll, Q, sg, &oi, &li) || !mi_piece(Ll, Q2, sg, &oo, &lo)) continue;
          const int s_in = Ll.pblk[Q][sg], s_out = Ll.pblk[Q2][sg];
          const int x = B.by_in[size_t(lab) * nsB + s_in];
          if (x < 0) continue;
          DMRG_REQUIRE(B.blocks[x].so == s_out && B.sec.d[s_in] == li && B.sec.d[s_out] == lo,
                       DMRG_EINVAL, "internal: carried block does not fit its pieces");
          here.push_back(EmbedTask{B.blocks[x].off, int64_t(oo) * Din + oi, li, Din, lo, li, 1.0});
        }
      } else if (!cre) {
        int o1, l1;
        if (mi_piece(Ll, Q, 1, &o1, &l1))
          here.push_back(EmbedTask{-1, int64_t(o1) * Din + o1, 0, Din, l1, l1, 1.0});
      } else {
        int o0, l0, o1, l1;
        if (mi_piece(Ll, Q, 0, &o0, &l0) && mi_piece(Ll, Q2, 1, &o1, &l1)) {
          DMRG_REQUIRE(Ll.pblk[Q][0] == Ll.pblk[Q2][1] && l0 == l1, DMRG_EINVAL,
                       "internal: creation pieces differ");
          const QN qb = B.sec.q[Ll.pblk[Q][0]];
          here.push_back(EmbedTask{-1, int64_t(o1) * Din + o0, 0, Din, l1, l0,
                                   ((qb.a + qb.b) & 1) ? -1.0 : 1.0});
        }
      }
      if (here.empty()) continue;
      for (EmbedTask& t : here) {
        DMRG_REQUIRE(t.nc <= t.ldd && t.dst + int64_t(t.nr - 1) * t.ldd + t.nc <= int64_t(Dout) * Din &&
                         (t.src < 0 || t.src + int64_t(t.nr - 1) * t.lds + t.nc <= B.n_elems),
                     DMRG_EINVAL, "internal: embedded block out of range");
        t.dst += eoff;
        emb.push_back(t);
      }
      E.blocks.push_back(OpBlock{Q2, Q, eoff});
      eoff += int64_t(Dout) * Din;
    }
  }
  E.lab_ptr[E.nlab] = int64_t(E.blocks.size());
  E.n_elems = eoff;
  E.data.alloc(std::max<int64_t>(eoff, 1));
  DMRG_CUDA(cudaMemsetAsync(E.data.p, 0, sizeof(double) * std::max<int64_t>(eoff, 1), c.stream));
  DevBuf<EmbedTask> de;
  de.upload(emb, c.stream);
  embed_blocks(de.p, int64_t(emb.size()), B.data.p, E.data.p, c.stream);
  E.index_by_in();
  OpSet out;
  project(c, E, iso, out);
  sync(c);
  mr.ops = std::move(out);
}

static void step(Ctx& c, int p, int dir, int M, dmrg_step_stats* st,
                 double* late_energy = nullptr, MiRun* mi = nullptr) {
  double t0 = now_s();
  Super& sb = super_at(c, p);
  // the block that the next step of this sweep enlarges on the side this step leaves as
  // it is: plan its enlargement on a host thread while the GPU runs this step
  if (dir == 0 && p + 2 <= c.N - 2 && c.right[p + 2].valid)
    start_prefetch(c, c.right[p + 2].ops, c.right[p + 2].gen, p + 2, false);
  else if (dir == 1 && p - 2 >= 0 && c.left[p - 2].valid)
    start_prefetch(c, c.left[p - 2].ops, c.left[p - 2].gen, p - 1, true);
  c.psi_guess.alloc(std::max<int64_t>(sb.size, 1));
  const bool two = c.n_roots == 2;
  const bool pred1 = two && c.psi1_valid && c.psi_valid && c.prev;
  if (pred1) {   // White's prediction of the second state through the same bases
    c.psi_guess1.alloc(std::max<int64_t>(sb.size, 1));
    predict(c, sb, p, dir, c.psi_guess1.p, c.psi1.p);
  }
  predict(c, sb, p, dir, c.psi_guess.p);
  c.psi.alloc(std::max<int64_t>(sb.size, 1));
  if (two) c.psi1.alloc(std::max<int64_t>(sb.size, 1));
  settle_energy(c);   // the previous step's energy (its product reads vectors Davidson reuses)
  c.psi1_valid = false;
  DavResult r = davidson(c, sb, c.psi_guess.p, c.psi.p, true, pred1 ? c.psi_guess1.p : nullptr,
                         two ? c.psi1.p : nullptr);
  DMRG_REQUIRE(!two || !std::isnan(r.theta1), DMRG_EINVAL,
               "the superblock holds fewer states than the two targeted ones");
  c.psi1_valid = two;
  if (dir == 0 && p + 2 <= c.N - 2 && c.right[p + 2].valid) issue_prefetch_device(c, c.right[p + 2].ops);
  else if (dir == 1 && p - 2 >= 0 && c.left[p - 2].valid) issue_prefetch_device(c, c.left[p - 2].ops);
  const double flops = sb.flops, bytes = sb.bytes;
  c.psi_valid = true;
  c.psi_p = p;
  if (mi) mi_measure(c, *mi, sb, p);
  TruncResult tr = truncate_renormalize(c, p, dir, M);   // overlaps the Rayleigh quotient
  if (mi) mi_carry(c, *mi, sb, p);
  const bool late = late_energy && c.rq_pending;
  if (!late) dav_energy(c, r);
  if (st) {
    st->p = p;
    st->dir = dir;
    st->n_products = r.nprod;
    st->kept = tr.kept;
    st->energy = r.theta;
    st->residual = std::max(r.resid, r.resid1);
    st->trunc_err = tr.trunc;
    st->seconds = now_s() - t0;
    st->energy1 = r.theta1;
    st->heff_seconds = r.heff_seconds;
    st->heff_flops = flops;
    st->heff_bytes = bytes;
  }
  if (late) {
    launch_rq(c);
    c.rq_target = late_energy;
  }
}

bool heff_view(dmrg_ctx* c, int p, HeffView* v) {
  if (!c || !c->sb || c->sb->p != p) return false;
  Super& sb = *c->sb;
  v->st1 = &sb.st1;
  v->st2 = &sb.st2;
  v->L = sb.L.data.p;
  v->R = sb.R.data.p;
  v->size = sb.size;
  v->t_elems = sb.t_elems;
  v->stream = c->stream;
  v->device = c->device;
  v->lists_ready = sb.two_stage_ready;
  return true;
}

void set_error(dmrg_ctx* c, const char* msg) {
  if (c) c->err = msg;
}

}  // namespace dmrg

// =======================================================================================
// C-ABI
// =======================================================================================
using namespace dmrg;

template <class F>
static int guarded(dmrg_ctx* c, F&& f) {
  if (!c) return DMRG_EINVAL;
  struct PoolScope {
    Pool* prev;
    explicit PoolScope(Pool* p) : prev(tl_pool) { tl_pool = p; }
    ~PoolScope() { tl_pool = prev; }
  } scope(&c->pool);
  try {
    f();
    return DMRG_OK;
  } catch (const Error& e) {
    c->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return DMRG_ENOMEM;
  } catch (const std::exception& e) {
    c->err = e.what();
    return DMRG_EINVAL;
  }
}

// Host tables of the bookkeeping (tens of MB per step at large M) are allocated and freed
// every step; glibc would return such blocks to the kernel and page them in again.  Keep
// blocks up to 32 MB in the heap and never trim it, once per process.
static void tune_host_allocator() {
  static std::once_flag once;
  std::call_once(once, [] {
    mallopt(M_MMAP_THRESHOLD, 32 << 20);
    mallopt(M_TRIM_THRESHOLD, 1 << 30);
  });
}

extern "C" int dmrg_create(const dmrg_problem* prob, const dmrg_options* opt, dmrg_ctx** out) {
  if (!out) return DMRG_EINVAL;
  *out = nullptr;
  dmrg_ctx* c = nullptr;
  try {
    c = new dmrg_ctx();
  } catch (...) {
    return DMRG_ENOMEM;
  }
  tune_host_allocator();
  int st = guarded(c, [&] {
    DMRG_REQUIRE(opt != nullptr, DMRG_EINVAL, "options are NULL");
    c->opt = *opt;
    DMRG_REQUIRE(opt->precision == DMRG_FP64 || opt->precision == DMRG_MIXED_FP32, DMRG_EINVAL,
                 "unknown precision");
    DMRG_REQUIRE(opt->dav_tol > 0 && opt->dav_max_iter >= 1 && opt->dav_max_sub >= 4 &&
                     opt->dav_max_sub <= 64,
                 DMRG_EINVAL, "bad Davidson options");
    c->stream = static_cast<cudaStream_t>(opt->stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) {   // no device here: host-only use
      c->device = -1;
      (void)cudaGetLastError();
    }
    build_chain(prob, c->chain);
    c->order.assign(prob->order, prob->order + c->chain.N);
    build_mpo(c->chain, c->mpo);
    c->N = c->chain.N;
    build_reach(*c);
    c->w_by_b.resize(c->N);
    c->w_by_a.resize(c->N);
    c->ent_left.resize(c->N);
    c->ent_right.resize(c->N);
    for (int s = 0; s < c->N; ++s) {
      const auto& W = c->mpo.W[s];
      std::vector<int> idx(W.size());
      for (size_t i = 0; i < W.size(); ++i) idx[i] = int(i);
      c->w_by_b[s] = idx;
      std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return W[x].a < W[y].a; });
      c->w_by_a[s] = idx;
      for (size_t i = 1; i < W.size(); ++i)
        DMRG_REQUIRE(W[i].b >= W[i - 1].b, DMRG_EINVAL, "internal: entries not grouped");
    }
  });
  if (st != DMRG_OK) {
    // keep the context so that the caller can read the message, as documented
    *out = c;
    return st;
  }
  *out = c;
  return DMRG_OK;
}

extern "C" int dmrg_destroy(dmrg_ctx* c) {
  if (!c) return DMRG_OK;
  delete c;
  return DMRG_OK;
}

extern "C" const char* dmrg_last_error(const dmrg_ctx* c) {
  return c ? c->err.c_str() : "NULL context";
}

extern "C" int dmrg_build_blocks(dmrg_ctx* c, const dmrg_mps_init* init) {
  return guarded(c, [&] {
    DMRG_REQUIRE(c->N > 0, DMRG_EINVAL, "context was not created successfully");
    build_blocks(*c, init);
  });
}

extern "C" int dmrg_psi_layout(dmrg_ctx* c, int32_t p, int64_t* n_blocks, int64_t* size,
                               int32_t* qn_left, int32_t* dl, int32_t* dr, int64_t* off) {
  return guarded(c, [&] {
    Super& sb = super_at(*c, p);
    ensure_two_stage(*c, sb);
    if (n_blocks) *n_blocks = int64_t(sb.bL.size());
    if (size) *size = sb.size;
    for (size_t b = 0; b < sb.bL.size(); ++b) {
      if (qn_left) {
        const QN& q = sb.Ll.sec.q[sb.bL[b]];
        qn_left[3 * b] = q.a;
        qn_left[3 * b + 1] = q.b;
        qn_left[3 * b + 2] = q.m;
      }
      if (dl) dl[b] = sb.bdl[b];
      if (dr) dr[b] = sb.bdr[b];
      if (off) off[b] = sb.boff[b];
    }
  });
}

extern "C" int dmrg_heff_apply(dmrg_ctx* c, int32_t p, const double* x, double* y) {
  return guarded(c, [&] {
    DMRG_REQUIRE(x && y && x != y, DMRG_EINVAL, "bad vectors");
    Super& sb = super_at(*c, p);
    ensure_two_stage(*c, sb);
    heff(*c, sb, x, y, c->stream);
    sync(*c);
  });
}

extern "C" int dmrg_davidson(dmrg_ctx* c, int32_t p, const double* guess, double* out,
                             double* energy, dmrg_dav_stats* st) {
  int conv = 1;
  int rc = guarded(c, [&] {
    double t0 = now_s();
    Super& sb = super_at(*c, p);
    c->psi_guess.alloc(std::max<int64_t>(sb.size, 1));
    const int pdir = (c->prev && c->prev->p > p) ? 1 : 0;
    const bool two = c->n_roots == 2;
    const bool pred1 = two && !guess && c->psi1_valid && c->psi_valid && c->prev;
    if (pred1) {
      c->psi_guess1.alloc(std::max<int64_t>(sb.size, 1));
      predict(*c, sb, p, pdir, c->psi_guess1.p, c->psi1.p);
    }
    if (guess) {
      DMRG_CUDA(cudaMemcpyAsync(c->psi_guess.p, guess, sizeof(double) * sb.size,
                                cudaMemcpyDeviceToDevice, c->stream));
    } else {
      predict(*c, sb, p, pdir, c->psi_guess.p);
    }
    c->psi.alloc(std::max<int64_t>(sb.size, 1));
    if (two) c->psi1.alloc(std::max<int64_t>(sb.size, 1));
    c->psi1_valid = false;
    DavResult r = davidson(*c, sb, c->psi_guess.p, c->psi.p, false,
                           pred1 ? c->psi_guess1.p : nullptr, two ? c->psi1.p : nullptr);
    DMRG_REQUIRE(!two || !std::isnan(r.theta1), DMRG_EINVAL,
                 "the superblock holds fewer states than the two targeted ones");
    c->psi_valid = true;
    c->psi1_valid = two;
    c->psi_p = p;
    if (out) {
      DMRG_CUDA(cudaMemcpyAsync(out, c->psi.p, sizeof(double) * sb.size, cudaMemcpyDeviceToDevice,
                                c->stream));
      sync(*c);
    }
    if (energy) *energy = r.theta;
    if (st) {
      st->n_products = r.nprod;
      st->converged = r.converged ? 1 : 0;
      st->residual = std::max(r.resid, r.resid1);
      st->energy = r.theta;
      st->heff_flops = sb.flops;
      st->heff_bytes = sb.bytes;
      st->seconds = now_s() - t0;
      st->energy1 = r.theta1;
    }
    conv = r.converged ? 1 : 0;
  });
  if (rc == DMRG_OK && !conv) {
    c->err = "Davidson did not reach the tolerance within dav_max_iter products";
    return DMRG_ENOCONV;
  }
  return rc;
}

extern "C" int dmrg_truncate_renormalize(dmrg_ctx* c, int32_t p, int32_t dir, int32_t M,
                                         double* trunc_err, int32_t* kept) {
  return guarded(c, [&] {
    TruncResult tr = truncate_renormalize(*c, p, dir, M);
    if (trunc_err) *trunc_err = tr.trunc;
    if (kept) *kept = tr.kept;
    DMRG_REQUIRE(!tr.noconv, DMRG_ENOCONV,
                 "a density-matrix eigendecomposition stopped at its sweep limit (result "
                 "installed)");
  });
}

extern "C" int dmrg_rdm_eigh(dmrg_ctx* c, int32_t p, int32_t dir, int32_t cluster,
                             int32_t* n_sec, int64_t* size, int32_t* qn, int32_t* dims,
                             double* w, double* vecs) {
  return guarded(c, [&] {
    DMRG_REQUIRE(c->psi_valid && c->psi_p == p, DMRG_EINVAL,
                 "no wave function held for this position (run dmrg_davidson or dmrg_step)");
    DMRG_REQUIRE(dir == 0 || dir == 1, DMRG_EINVAL, "dir must be 0 or 1");
    DMRG_REQUIRE(cluster == 0 || cluster == 1 || cluster == 8 || cluster == 16, DMRG_EINVAL,
                 "cluster must be 0, 1, 8 or 16");
    DMRG_REQUIRE(c->n_roots == 1 || c->psi1_valid, DMRG_EINVAL,
                 "no second targeted state held for this position");
    Super* sb = (c->sb && c->sb->p == p) ? c->sb.get()
                                          : (c->prev && c->prev->p == p ? c->prev.get() : nullptr);
    DMRG_REQUIRE(sb != nullptr, DMRG_EINVAL, "the layout of the held wave function is gone");
    const Layout& lay = dir == 0 ? sb->Ll : sb->Rl;
    const RdmLayout RL = rdm_layout(lay);
    if (n_sec) *n_sec = RL.ns;
    if (size) *size = RL.sq;
    if (!qn && !dims && !w && !vecs) return;
    const bool noconv = rdm_eigh(*c, *sb, dir, RL, cluster);
    for (int i = 0; i < RL.ns; ++i) {
      if (qn) {
        qn[3 * i] = lay.sec.q[i].a;
        qn[3 * i + 1] = lay.sec.q[i].b;
        qn[3 * i + 2] = lay.sec.q[i].m;
      }
      if (dims) dims[i] = RL.dims[i];
    }
    if (w && RL.total)
      DMRG_CUDA(cudaMemcpyAsync(w, c->ew.p, sizeof(double) * RL.total, cudaMemcpyDeviceToHost,
                                c->stream));
    if (vecs && RL.sq)
      DMRG_CUDA(cudaMemcpyAsync(vecs, c->eVs.p, sizeof(double) * RL.sq, cudaMemcpyDeviceToHost,
                                c->stream));
    sync(*c);
    DMRG_REQUIRE(!noconv, DMRG_ENOCONV,
                 "a density-matrix eigendecomposition stopped at its sweep limit");
  });
}

extern "C" int dmrg_dot_rdm(dmrg_ctx* c, int32_t p, double* rho, double* ent) {
  return guarded(c, [&] {
    DMRG_REQUIRE(c->psi_valid && c->psi_p == p, DMRG_EINVAL,
                 "no wave function held for this position (run dmrg_davidson or dmrg_step)");
    Super* sb = (c->sb && c->sb->p == p) ? c->sb.get()
                                          : (c->prev && c->prev->p == p ? c->prev.get() : nullptr);
    DMRG_REQUIRE(sb != nullptr, DMRG_EINVAL, "the layout of the held wave function is gone");
    const Layout& Ll = sb->Ll;
    const Layout& Rl = sb->Rl;
    // rows (columns) of piece sigma of an enlarged sector: pieces are contiguous, state 0 first
    auto extent = [](const Layout& L, int Q, int sg, int* off, int* len) {
      if (L.pblk[Q][sg] < 0) return false;
      const int D = L.sec.d[Q];
      *off = L.poff[Q][sg];
      *len = (sg == 0 && L.pblk[Q][1] >= 0 ? L.poff[Q][1] : D) - *off;
      return *len > 0;
    };
    std::vector<RdmTask> tasks;
    for (size_t b = 0; b < sb->bL.size(); ++b) {
      const int QL = sb->bL[b], QR = sb->bR[b], dR = sb->bdr[b];
      for (int sl = 0; sl < 2; ++sl)
        for (int sr = 0; sr < 2; ++sr) {
          int ro, nr, co, nc;
          if (!extent(Ll, QL, sl, &ro, &nr) || !extent(Rl, QR, sr, &co, &nc)) continue;
          const int64_t a = sb->boff[b] + int64_t(ro) * dR + co;
          tasks.push_back(RdmTask{a, a, dR, dR, nr, nc, 2 * sl + sr, 0});
        }
    }
    // the hop between dots of equal quantum numbers: psi(l, 1, 0, r) psi(l, 0, 1, r)
    const QN qs = c->chain.q[p];
    if (qs == c->chain.q[p + 1]) {
      for (size_t b = 0; b < sb->bL.size(); ++b) {
        const int QL = sb->bL[b], QR = sb->bR[b], dR = sb->bdr[b];
        int ro, nr, co, nc;
        if (!extent(Ll, QL, 1, &ro, &nr) || !extent(Rl, QR, 0, &co, &nc)) continue;
        const int QL2 = Ll.sec.find(Ll.sec.q[QL] - qs);
        if (QL2 < 0 || Ll.pblk[QL2][0] != Ll.pblk[QL][1]) continue;
        const int b2 = sb->psi_of_L[QL2];
        if (b2 < 0) continue;
        const int QR2 = sb->bR[b2];
        if (Rl.sec.q[QR2] != Rl.sec.q[QR] + qs || Rl.pblk[QR2][1] != Rl.pblk[QR][0]) continue;
        int ro2, nr2, co2, nc2;
        if (!extent(Ll, QL2, 0, &ro2, &nr2) || !extent(Rl, QR2, 1, &co2, &nc2)) continue;
        DMRG_REQUIRE(nr2 == nr && nc2 == nc, DMRG_EINVAL, "internal: hop pieces differ in size");
        const int dR2 = sb->bdr[b2];
        tasks.push_back(RdmTask{sb->boff[b] + int64_t(ro) * dR + co,
                                sb->boff[b2] + int64_t(ro2) * dR2 + co2, dR, dR2, nr, nc, 4, 0});
      }
    }
    for (const RdmTask& t : tasks)   // every piece inside the wave function
      DMRG_REQUIRE(t.a >= 0 && t.b >= 0 && t.a + int64_t(t.nr - 1) * t.lda + t.nc <= sb->size &&
                       t.b + int64_t(t.nr - 1) * t.ldb + t.nc <= sb->size,
                   DMRG_EINVAL, "internal: density-matrix piece outside the wave function");
    DevBuf<RdmTask> dt;
    DevBuf<double> part, sums;
    dt.upload(tasks, c->stream);
    part.alloc(std::max<int64_t>(int64_t(tasks.size()), 1));
    sums.alloc(8);
    rdm_sums(dt.p, int64_t(tasks.size()), c->psi.p, part.p, sums.p, c->stream);
    double h[5];
    dav_readback(*c, sums.p, 5, h);
    double r[16] = {0};
    for (int k = 0; k < 4; ++k) r[5 * k] = h[k];
    r[6] = r[9] = h[4];
    if (rho) std::copy(r, r + 16, rho);
    if (ent) {
      auto vn = [](std::initializer_list<double> w) {
        double s = 0.0;
        for (double x : w)
          if (x > 0.0) s -= x * std::log(x);
        return s;
      };
      const double sp = vn({h[0] + h[1], h[2] + h[3]});
      const double sq = vn({h[0] + h[2], h[1] + h[3]});
      const double mid = 0.5 * (h[1] + h[2]);
      const double rad = std::sqrt(0.25 * (h[1] - h[2]) * (h[1] - h[2]) + h[4] * h[4]);
      const double spq = vn({h[0], h[3], mid + rad, mid - rad});
      ent[0] = sp;
      ent[1] = sq;
      ent[2] = spq;
      ent[3] = sp + sq - spq;
    }
  });
}

extern "C" int dmrg_set_roots(dmrg_ctx* c, int32_t n_roots) {
  return guarded(c, [&] {
    DMRG_REQUIRE(n_roots == 1 || n_roots == 2, DMRG_EINVAL, "n_roots must be 1 or 2");
    DMRG_REQUIRE(n_roots == 1 || (c->opt.precision == DMRG_FP64 &&
                                  c->opt.precond == DMRG_PRECOND_DIAG),
                 DMRG_EINVAL, "two-state targeting needs DMRG_FP64 and the diagonal preconditioner");
    if (n_roots != c->n_roots) c->psi1_valid = false;
    c->n_roots = n_roots;
  });
}

extern "C" int dmrg_set_dbss(dmrg_ctx* c, int32_t M_min, double trunc_target) {
  return guarded(c, [&] {
    DMRG_REQUIRE(trunc_target <= 0.0 || (M_min >= 1 && trunc_target < 1.0), DMRG_EINVAL,
                 "DBSS needs M_min >= 1 and 0 < trunc_target < 1");
    c->dbss_min = trunc_target > 0.0 ? M_min : 0;
    c->dbss_target = trunc_target > 0.0 ? trunc_target : 0.0;
  });
}

extern "C" int dmrg_step(dmrg_ctx* c, int32_t p, int32_t dir, int32_t M, dmrg_step_stats* st) {
  return guarded(c, [&] {
    DMRG_REQUIRE(dir == 0 || dir == 1, DMRG_EINVAL, "dir must be 0 or 1");
    step(*c, p, dir, M, st);
  });
}

extern "C" int dmrg_sweep(dmrg_ctx* c, int32_t M, dmrg_step_stats* steps, double* energy) {
  return guarded(c, [&] {
    DMRG_REQUIRE(c->built, DMRG_EINVAL, "dmrg_build_blocks has not been called");
    std::vector<dmrg_step_stats> all(2 * size_t(c->N - 3));
    int k = 0;
    try {
      for (int p = 1; p <= c->N - 3; ++p, ++k) step(*c, p, 0, M, &all[k], &all[k].energy);
      for (int p = c->N - 3; p >= 1; --p, ++k) step(*c, p, 1, M, &all[k], &all[k].energy);
      settle_energy(*c);
    } catch (...) {
      c->rq_target = nullptr;   // the stats are local to this call
      throw;
    }
    if (steps) std::copy(all.begin(), all.end(), steps);
    if (energy && !all.empty()) *energy = all.back().energy;
  });
}

extern "C" int dmrg_mutual_information(dmrg_ctx* c, int32_t M, double* I, double* s,
                                       dmrg_step_stats* steps) {
  return guarded(c, [&] {
    DMRG_REQUIRE(c->built, DMRG_EINVAL, "dmrg_build_blocks has not been called");
    DMRG_REQUIRE(I != nullptr && s != nullptr, DMRG_EINVAL, "NULL output");
    DMRG_REQUIRE(M >= 1, DMRG_EINVAL, "M must be positive");
    DMRG_REQUIRE(c->n_roots == 1, DMRG_EINVAL, "the mutual information is for one targeted state");
    const int N = c->N;
    MiRun mr;
    mr.N = N;
    mr.I.assign(size_t(N) * N, 0.0);
    mr.s.assign(size_t(N), 0.0);
    mi_init(*c, mr);
    std::vector<dmrg_step_stats> all(size_t(N - 3));
    for (int p = 1; p <= N - 3; ++p) step(*c, p, 0, M, &all[p - 1], nullptr, &mr);
    settle_energy(*c);
    if (steps) std::copy(all.begin(), all.end(), steps);
    for (int i = 0; i < N; ++i) {
      s[c->order[i]] = mr.s[i];
      for (int j = 0; j < N; ++j) I[size_t(c->order[i]) * N + c->order[j]] = mr.I[size_t(i) * N + j];
    }
  });
}

extern "C" int dmrg_block_sectors(dmrg_ctx* c, int32_t side, int32_t b, int32_t* n, int32_t* qn,
                                  int32_t* dims) {
  return guarded(c, [&] {
    DMRG_REQUIRE(b >= 0 && b < c->N && (side == 0 || side == 1), DMRG_EINVAL, "bad block");
    const Blk& B = side == 0 ? c->left[b] : c->right[b];
    DMRG_REQUIRE(B.valid, DMRG_EINVAL, "block not available");
    const SectorSet& s = B.ops.sec;
    if (n) *n = s.size();
    for (int i = 0; i < s.size(); ++i) {
      if (qn) {
        qn[3 * i] = s.q[i].a;
        qn[3 * i + 1] = s.q[i].b;
        qn[3 * i + 2] = s.q[i].m;
      }
      if (dims) dims[i] = s.d[i];
    }
  });
}

// drop the superblock held by the context (rebuilt at its next use), after any Rayleigh
// quotient still reading it
static void drop_superblock(Ctx& c) {
  if (!c.sb) return;
  settle_energy(c);
  if (c.rq_pending) {
    launch_rq(c);
    DMRG_CUDA(cudaEventSynchronize(c.rq_out));
  }
  DMRG_CUDA(cudaStreamSynchronize(c.stream));
  if (c.rq_sb == c.sb.get()) c.rq_sb = nullptr;
  c.sb.reset();
}

extern "C" int dmrg_set_options(dmrg_ctx* c, const dmrg_options* opt) {
  return guarded(c, [&] {
    DMRG_REQUIRE(opt != nullptr, DMRG_EINVAL, "options are NULL");
    DMRG_REQUIRE(opt->precision == DMRG_FP64 || opt->precision == DMRG_MIXED_FP32, DMRG_EINVAL,
                 "unknown precision");
    DMRG_REQUIRE(opt->dav_tol > 0 && opt->dav_max_iter >= 1 && opt->dav_max_sub >= 4 &&
                     opt->dav_max_sub <= 64,
                 DMRG_EINVAL, "bad Davidson options");
    DMRG_REQUIRE(c->n_roots == 1 || (opt->precision == DMRG_FP64 &&
                                     opt->precond == DMRG_PRECOND_DIAG),
                 DMRG_EINVAL, "two-state targeting needs DMRG_FP64 and the diagonal preconditioner");
    const bool prec_changed = opt->precision != c->opt.precision;
    // byte counts, FP32 operator shadows and product lists depend on the precision
    if (prec_changed) drop_superblock(*c);
    c->opt = *opt;
    c->stream = static_cast<cudaStream_t>(opt->stream);
  });
}

extern "C" int dmrg_set_tuning(dmrg_ctx* c, const dmrg_tuning* t) {
  return guarded(c, [&] {
    DMRG_REQUIRE(t != nullptr, DMRG_EINVAL, "NULL tuning");
    DMRG_REQUIRE(t->heff_big_edge >= 0 && t->heff_big_edge <= 4096, DMRG_EINVAL,
                 "heff_big_edge must lie in [0, 4096]");
    DMRG_REQUIRE(t->svd_cluster == 0 || t->svd_cluster == 1 || t->svd_cluster == 8 ||
                     t->svd_cluster == 16,
                 DMRG_EINVAL, "svd_cluster must be 0, 1, 8 or 16");
    DMRG_REQUIRE(t->heff_graph == 0 || t->heff_graph == 1, DMRG_EINVAL,
                 "heff_graph must be 0 or 1");
    c->big_edge = t->heff_big_edge;
    c->svd_cluster = t->svd_cluster;
    c->heff_graph = t->heff_graph;
    drop_superblock(*c);   // its product lists follow the old split: rebuilt at the next use
  });
}

extern "C" int dmrg_autotune(dmrg_ctx* c, int32_t p, int32_t reps, int32_t* chosen,
                             int32_t* edges, double* ms) {
  return guarded(c, [&] {
    DMRG_REQUIRE(reps >= 1, DMRG_EINVAL, "reps must be at least 1");
    static const int kCand[5] = {0, 32, 64, 128, 256};
    double best_ms[5];
    const int keep = c->big_edge;
    cudaEvent_t e0, e1;
    DMRG_CUDA(cudaEventCreate(&e0));
    DMRG_CUDA(cudaEventCreate(&e1));
    try {
      for (int i = 0; i < 5; ++i) {
        c->big_edge = kCand[i];
        drop_superblock(*c);
        Super& sb = super_at(*c, p);
        DevBuf<double> x, y;
        x.alloc(std::max<int64_t>(sb.size, 1));
        y.alloc(std::max<int64_t>(sb.size, 1));
        fill_value(x.p, sb.size, 1.0 / std::sqrt(double(std::max<int64_t>(sb.size, 1))),
                   c->stream);
        // untimed: first use of the lists and buffers, then the graph capture
        heff(*c, sb, x.p, y.p, c->stream);
        heff(*c, sb, x.p, y.p, c->stream);
        double bt = 1e300;
        for (int r = 0; r < reps; ++r) {
          DMRG_CUDA(cudaEventRecord(e0, c->stream));
          heff(*c, sb, x.p, y.p, c->stream);
          DMRG_CUDA(cudaEventRecord(e1, c->stream));
          DMRG_CUDA(cudaEventSynchronize(e1));
          float t = 0.f;
          DMRG_CUDA(cudaEventElapsedTime(&t, e0, e1));
          bt = std::min(bt, double(t));
        }
        best_ms[i] = bt;
      }
    } catch (...) {
      c->big_edge = keep;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int pick = 0;
    for (int i = 1; i < 5; ++i)
      if (best_ms[i] < best_ms[pick]) pick = i;
    for (int i = 1; i < 5; ++i)   // the smallest positive edge within 5 % of the fastest
      if (best_ms[i] <= 1.05 * best_ms[pick]) {
        pick = i;
        break;
      }
    c->big_edge = kCand[pick];
    drop_superblock(*c);
    if (chosen) *chosen = kCand[pick];
    for (int i = 0; i < 5; ++i) {
      if (edges) edges[i] = kCand[i];
      if (ms) ms[i] = best_ms[i];
    }
  });
}

extern "C" int dmrg_get_tuning(dmrg_ctx* c, dmrg_tuning* t) {
  return guarded(c, [&] {
    DMRG_REQUIRE(t != nullptr, DMRG_EINVAL, "NULL tuning");
    t->heff_big_edge = c->big_edge;
    t->svd_cluster = c->svd_cluster;
    t->heff_graph = c->heff_graph;
  });
}

extern "C" int dmrg_partition_terms(dmrg_ctx* c, int32_t b, int32_t* n_terms) {
  return guarded(c, [&] {
    DMRG_REQUIRE(n_terms != nullptr, DMRG_EINVAL, "NULL output");
    DMRG_REQUIRE(b >= 0 && b <= c->N - 2, DMRG_EINVAL, "bond out of range [0, N-2]");
    *n_terms = int32_t(c->mpo.labels[b + 1].size());
  });
}

extern "C" int dmrg_get_counters(dmrg_ctx* c, dmrg_counters* out) {
  return guarded(c, [&] {
    DMRG_REQUIRE(out != nullptr, DMRG_EINVAL, "NULL output");
    out->launches = g_launches.load();
    out->heff_products = c->heff_products;
    out->heff_seconds = c->heff_seconds;
    out->heff_flops = c->heff_flops;
    out->heff_bytes = c->heff_bytes;
    out->t_enlarge = c->t_enlarge;
    out->t_super = c->t_super;
    out->t_davidson = c->t_davidson;
    out->t_truncate = c->t_truncate;
    out->t_project = c->t_project;
    out->t_predict = c->t_predict;
    out->t_sync = c->t_sync;
    out->t_enlarge_host = c->t_enlarge_host;
    out->t_upload = 1e-9 * double(g_upload_ns.load());
    out->upload_bytes = g_upload_bytes.load();
    out->sb_blocks_l = c->last_sizes[0];
    out->sb_blocks_r = c->last_sizes[1];
    out->sb_terms = c->last_sizes[2];
    out->sb_tiles = c->last_sizes[3];
    out->sb_small_tiles = c->last_sizes[4];
    for (int i = 0; i < 8; ++i) out->sb_term_hist[i] = c->term_hist[i];
    out->sb_kernel_flops = c->kernel_flops;
    for (int i = 0; i < 24; ++i) out->t_detail[i] = c->t_detail[i];
    out->t_detail[15] = 1e-9 * double(g_malloc_ns.load());
    out->t_detail[21] = double(c->eig_noconv);
    out->t_detail[22] = double(c->graph_replays);
    out->pool_mallocs = g_malloc_count.load();
  });
}

static uint64_t splitmix(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void mlp_init(Ctx& c, uint64_t seed) {
  const int64_t np = mlp_n_params();
  std::vector<float> h(np, 0.0f);
  // He-normal weights (Box-Muller on SplitMix64), zero biases
  const int64_t sizes[4][3] = {{0, 256, 4}, {256 * 4 + 256, 256, 256},
                               {256 * 4 + 256 + 256 * 256 + 256, 256, 256},
                               {256 * 4 + 256 + 2 * (256 * 256 + 256), 1, 256}};
  uint64_t st = seed;
  for (auto& L : sizes) {
    const double sd = std::sqrt(2.0 / double(L[2]));
    for (int64_t i = 0; i < L[1] * L[2]; ++i) {
      const double u1 = (splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      const double u2 = (splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      h[L[0] + i] = float(sd * std::sqrt(-2.0 * std::log(1.0 - u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  c.mlp_p.upload(h, c.stream);
  c.mlp_g.alloc(np);
  c.mlp_m.alloc(np);
  c.mlp_v.alloc(np);
  DMRG_CUDA(cudaMemsetAsync(c.mlp_m.p, 0, sizeof(float) * np, c.stream));
  DMRG_CUDA(cudaMemsetAsync(c.mlp_v.p, 0, sizeof(float) * np, c.stream));
  sync(c);
  c.mlp_ready = true;
  c.mlp_trained = false;
  c.mlp_step = 0;
}

extern "C" int dmrg_mlp_reset(dmrg_ctx* c, uint64_t seed) {
  return guarded(c, [&] { mlp_init(*c, seed); });
}

extern "C" int dmrg_mlp_harvest(dmrg_ctx* c, int32_t enable, int32_t per_iter) {
  return guarded(c, [&] {
    DMRG_REQUIRE(per_iter >= 1, DMRG_EINVAL, "per_iter must be positive");
    c->mlp_harvest = enable ? 1 : 0;
    c->mlp_per_iter = per_iter;
  });
}

extern "C" int dmrg_mlp_train(dmrg_ctx* c, int32_t epochs, int32_t batch, double lr, uint64_t seed,
                              double* loss_out, int64_t* n_samples) {
  return guarded(c, [&] {
    DMRG_REQUIRE(epochs >= 0 && batch >= 1 && lr > 0, DMRG_EINVAL, "bad training parameters");
    DMRG_REQUIRE(c->mlp_nsamp > 0, DMRG_EINVAL, "no harvested samples");
    if (!c->mlp_ready) mlp_init(*c, seed);
    const int64_t ns = c->mlp_nsamp, np = mlp_n_params();
    const int64_t B = std::min<int64_t>(batch, ns);
    c->mlp_X.alloc(B * 4);
    c->mlp_T.alloc(B);
    c->mlp_idx.alloc(ns);
    std::vector<int32_t> perm(ns);
    uint64_t st = seed ^ 0x5DEECE66Dull;
    double last = 0.0;
    for (int e = 0; e < epochs; ++e) {
      for (int64_t i = 0; i < ns; ++i) perm[i] = int32_t(i);
      for (int64_t i = ns - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(st) % uint64_t(i + 1)]);
      c->mlp_idx.upload(perm, c->stream);
      double tot = 0.0;
      int nbat = 0;
      for (int64_t b0 = 0; b0 + B <= ns; b0 += B) {
        mlp_gather<float>(c->mlp_samples.p, c->mlp_idx.p + b0, B, c->mlp_X.p, c->mlp_T.p, c->stream);
        mlp_forward<float>(c->mlp_p.p, c->mlp_X.p, B, c->mlp_acts, c->stream);
        tot += mlp_backward<float>(c->mlp_p.p, c->mlp_X.p, c->mlp_T.p, B, c->mlp_acts, c->mlp_g.p,
                                   c->stream);
        ++nbat;
        mlp_adam<float>(c->mlp_p.p, c->mlp_g.p, c->mlp_m.p, c->mlp_v.p, np, lr, ++c->mlp_step,
                        c->stream);
      }
      last = nbat ? tot / nbat : 0.0;
    }
    sync(*c);
    c->mlp_trained = true;
    if (loss_out) *loss_out = last;
    if (n_samples) *n_samples = ns;
  });
}

extern "C" int dmrg_mlp_params(dmrg_ctx* c, int32_t dir, double* host, int64_t n) {
  return guarded(c, [&] {
    const int64_t np = mlp_n_params();
    DMRG_REQUIRE(host && n == np, DMRG_EINVAL, "parameter buffer must hold dmrg_mlp_n_params()");
    std::vector<float> f(np);
    if (dir == 0) {
      DMRG_REQUIRE(c->mlp_ready, DMRG_EINVAL, "network not initialised");
      DMRG_CUDA(cudaMemcpyAsync(f.data(), c->mlp_p.p, sizeof(float) * np, cudaMemcpyDeviceToHost,
                                c->stream));
      sync(*c);
      for (int64_t i = 0; i < np; ++i) host[i] = f[i];
    } else {
      if (!c->mlp_ready) mlp_init(*c, 1);
      for (int64_t i = 0; i < np; ++i) f[i] = float(host[i]);
      c->mlp_p.upload(f, c->stream);
      sync(*c);
      c->mlp_trained = true;
    }
  });
}

template <class T>
static double loss_grad_t(Ctx& c, const double* P, const double* X, const double* Tg, int64_t B,
                          double* grad) {
  const int64_t np = mlp_n_params();
  std::vector<T> hp(P, P + np), hx(X, X + B * 4), ht(Tg, Tg + B), hg(np);
  DevBuf<T> dp, dx, dt, dg;
  dp.upload(hp, c.stream);
  dx.upload(hx, c.stream);
  dt.upload(ht, c.stream);
  dg.alloc(np);
  MlpActs<T> a;
  mlp_forward<T>(dp.p, dx.p, B, a, c.stream);
  const double loss = mlp_backward<T>(dp.p, dx.p, dt.p, B, a, dg.p, c.stream);
  DMRG_CUDA(cudaMemcpyAsync(hg.data(), dg.p, sizeof(T) * np, cudaMemcpyDeviceToHost, c.stream));
  sync(c);
  for (int64_t i = 0; i < np; ++i) grad[i] = double(hg[i]);
  return loss;
}

extern "C" int dmrg_mlp_loss_grad(dmrg_ctx* c, int32_t precision, const double* params,
                                  const double* X, const double* Tg, int64_t B, double* loss,
                                  double* grad) {
  return guarded(c, [&] {
    DMRG_REQUIRE(params && X && Tg && grad && B >= 1, DMRG_EINVAL, "bad arguments");
    double l = precision == DMRG_FP64 ? loss_grad_t<double>(*c, params, X, Tg, B, grad)
                                      : loss_grad_t<float>(*c, params, X, Tg, B, grad);
    if (loss) *loss = l;
  });
}

extern "C" int64_t dmrg_mlp_n_params(void) { return mlp_n_params(); }

extern "C" int dmrg_heff_cost(dmrg_ctx* c, int32_t p, double* flops, double* bytes,
                              int64_t* n_items) {
  return guarded(c, [&] {
    Super& sb = super_at(*c, p);
    if (flops) *flops = sb.flops;
    if (bytes) *bytes = sb.bytes;
    if (n_items) *n_items = sb.n_items;
  });
}

// =======================================================================================
// batch mode: several independent problems, one fused H_eff launch per Davidson iteration
// =======================================================================================
struct dmrg_batch {
  std::string err = "no error";
  std::vector<dmrg_ctx*> ctx;
  int precision = DMRG_FP64;
  cudaStream_t bs = nullptr;                 // internal stream (graph capture)
  cudaEvent_t ev = nullptr;
  std::vector<cudaEvent_t> ev_ctx;
  // combined lists of the current step
  dmrg::DevBuf<dmrg::HeffItem> items;
  dmrg::DevBuf<dmrg::HeffTile> tiles, stiles;
  dmrg::DevBuf<dmrg::HeffRed> red;
  int64_t n_tiles = 0, n_stiles = 0, n_red = 0;
  // per-iteration tables: input and output vector pointers, active flags
  struct Tab {
    const double* in[dmrg::kMaxInst];
    double* out[dmrg::kMaxInst];
    int32_t active[dmrg::kMaxInst];
  };
  Tab* h_tab = nullptr;                      // pinned
  Tab* d_tab = nullptr;
  cudaGraphExec_t exec = nullptr;
  int iter = 0;
  // counters
  int64_t products = 0, launches0 = 0;
  double heff_seconds = 0;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  ~dmrg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (h_tab) cudaFreeHost(h_tab);
    if (d_tab) cudaFree(d_tab);
    if (ev) cudaEventDestroy(ev);
    for (auto e : ev_ctx) cudaEventDestroy(e);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (bs) cudaStreamDestroy(bs);
  }
};

namespace dmrg {

struct PoolScope {
  Pool* prev;
  explicit PoolScope(Pool* p) : prev(tl_pool) { tl_pool = p; }
  ~PoolScope() { tl_pool = prev; }
};

// concatenate the fused lists of the instances' current superblocks (heaviest tiles first)
static void batch_lists(dmrg_batch& B, const std::vector<int>& inst) {
  std::vector<HeffItem> fi;
  std::vector<std::pair<double, HeffTile>> ft, fts;
  std::vector<HeffRed> fr;
  for (int i : inst) {
    Super& sb = *B.ctx[i]->sb;
    const int base = int(fi.size());
    fi.insert(fi.end(), sb.h_items.begin(), sb.h_items.end());
    auto add = [&](const std::vector<HeffTile>& tiles, const std::vector<double>& cost,
                   std::vector<std::pair<double, HeffTile>>& dst) {
      for (size_t t = 0; t < tiles.size(); ++t) {
        HeffTile x = tiles[t];
        x.i0 += base;
        x.i1 += base;
        x.inst = i;
        dst.push_back({cost[t], x});
      }
    };
    add(sb.h_tiles, sb.h_cost, ft);
    add(sb.h_stiles, sb.h_scost, fts);
    for (HeffRed r : sb.h_red) {
      r.inst = i;
      fr.push_back(r);
    }
  }
  auto sorted = [](std::vector<std::pair<double, HeffTile>>& v) {
    std::stable_sort(v.begin(), v.end(),
                     [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<HeffTile> tl(v.size());
    for (size_t t = 0; t < v.size(); ++t) tl[t] = v[t].second;
    return tl;
  };
  const std::vector<HeffTile> tl = sorted(ft), tls = sorted(fts);
  B.items.upload(fi, B.bs);
  B.tiles.upload(tl, B.bs);
  B.stiles.upload(tls, B.bs);
  B.red.upload(fr, B.bs);
  B.n_tiles = int64_t(tl.size());
  B.n_stiles = int64_t(tls.size());
  B.n_red = int64_t(fr.size());
  DMRG_CUDA(cudaStreamSynchronize(B.bs));
}

// the product sequence of one batched iteration on the internal stream: psi of every
// instance into its staging copy, one fused launch, one reduction, results out
static void batch_issue(dmrg_batch& B, const std::vector<int>& inst) {
  const int32_t* act = B.d_tab->active;
  if (B.precision == DMRG_FP64) {
    HeffPtrs<double> ptr{};
    ptr.active = act;
    for (int i : inst) {
      Ctx& c = *B.ctx[i];
      Super& sb = *c.sb;
      pad_psi_ind<double>(&B.d_tab->in[i], c.xpad64.p, sb.d_src_off.p, sb.d_pad_off.p,
                          sb.d_pad_len.p, int(sb.bL.size()), act + i, B.bs);
      ptr.L[i] = sb.L.data.p;
      ptr.R[i] = sb.R.data.p;
      ptr.X[i] = c.xpad64.p;
      ptr.Y[i] = c.ybat64.p;
      ptr.P[i] = c.part64.p;
    }
    heff_small<double>(B.stiles.p, B.n_stiles, B.items.p, ptr, B.bs);
    heff_fused<double>(B.tiles.p, B.n_tiles, B.items.p, B.red.p, B.n_red, ptr, B.bs);
    for (int i : inst) {   // big output blocks: grouped GEMM passes per instance
      Ctx& c = *B.ctx[i];
      Super& sb = *c.sb;
      if (!sb.n_big_blocks) continue;
      Bases<double> bb{};
      bb.p[B_LOPS] = sb.L.data.p;
      bb.p[B_ROPS] = sb.R.data.p;
      bb.p[B_X] = c.xpad64.p;
      bb.p[B_Y] = c.ybat64.p;
      bb.p[B_T] = c.T.p;
      bb.p[B_Z] = c.bigpart64.p;
      run_gemm_tasks<double>(sb.big1, bb, 1, B.bs, act + i);
      run_gemm_tasks<double>(sb.big2, bb, 1, B.bs, act + i);
      HeffPtrs<double> rp{};
      rp.Y[0] = c.ybat64.p;
      rp.P[0] = c.bigpart64.p;
      rp.active = act + i;
      heff_reduce<double>(sb.big_red.p, sb.n_big_red, rp, B.bs);
    }
    for (int i : inst) {
      Ctx& c = *B.ctx[i];
      out_to_f64_ind<double>(c.ybat64.p, &B.d_tab->out[i], c.sb->size, act + i, B.bs);
    }
  } else {
    HeffPtrs<float> ptr{};
    ptr.active = act;
    for (int i : inst) {
      Ctx& c = *B.ctx[i];
      Super& sb = *c.sb;
      pad_psi_ind<float>(&B.d_tab->in[i], c.xpad32.p, sb.d_src_off.p, sb.d_pad_off.p,
                         sb.d_pad_len.p, int(sb.bL.size()), act + i, B.bs);
      ptr.L[i] = sb.L.data32.p;
      ptr.R[i] = sb.R.data32.p;
      ptr.X[i] = c.xpad32.p;
      ptr.Y[i] = c.f32b.p;
      ptr.P[i] = c.part32.p;
    }
    heff_small<float>(B.stiles.p, B.n_stiles, B.items.p, ptr, B.bs);
    heff_tc(B.tiles.p, B.n_tiles, B.items.p, B.red.p, B.n_red, ptr, B.bs);
    for (int i : inst) {   // big output blocks: grouped GEMM passes per instance
      Ctx& c = *B.ctx[i];
      Super& sb = *c.sb;
      if (!sb.n_big_blocks) continue;
      Bases<void> bb{};
      bb.p[B_LOPS] = sb.L.data32.p;
      bb.p[B_ROPS] = sb.R.data32.p;
      bb.p[B_X] = c.xpad32.p;
      bb.p[B_Y] = c.f32b.p;
      bb.p[B_T] = c.f32T.p;
      bb.p[B_Z] = c.bigpart32.p;
      run_gemm_tasks_tc<float, float, float>(sb.big1, bb, 1, B.bs, act + i);
      run_gemm_tasks_tc<float, float, float>(sb.big2, bb, 1, B.bs, act + i);
      HeffPtrs<float> rp{};
      rp.Y[0] = c.f32b.p;
      rp.P[0] = c.bigpart32.p;
      rp.active = act + i;
      heff_reduce<float>(sb.big_red.p, sb.n_big_red, rp, B.bs);
    }
    for (int i : inst) {
      Ctx& c = *B.ctx[i];
      out_to_f64_ind<float>(c.f32b.p, &B.d_tab->out[i], c.sb->size, act + i, B.bs);
    }
  }
}

// staging buffers of every instance sized for its current superblock (before any capture)
static void batch_buffers(dmrg_batch& B, const std::vector<int>& inst) {
  for (int i : inst) {
    Ctx& c = *B.ctx[i];
    PoolScope ps(&c.pool);
    Super& sb = *c.sb;
    if (B.precision == DMRG_FP64) {
      c.part64.alloc(std::max<int64_t>(sb.p_elems, 1));
      c.xpad64.alloc(sb.pad_size);
      c.ybat64.alloc(std::max<int64_t>(sb.size, 1));
      if (sb.n_big_blocks) {
        c.T.alloc(std::max<int64_t>(sb.big_t_elems, 1));
        c.bigpart64.alloc(std::max<int64_t>(sb.big_p_elems, 1));
      }
    } else {
      c.f32b.alloc(std::max<int64_t>(sb.size, 1));
      c.part32.alloc(std::max<int64_t>(sb.p_elems, 1));
      c.xpad32.alloc(sb.pad_size);
      if (sb.n_big_blocks) {
        c.f32T.alloc(std::max<int64_t>(sb.big_t_elems, 1));
        c.bigpart32.alloc(std::max<int64_t>(sb.big_p_elems, 1));
      }
    }
  }
}

// one batched product: tables up, fused sequence (eager on the first iteration of a step,
// then captured once into a CUDA graph and replayed), ordering with every context stream
static void batch_product(dmrg_batch& B, const std::vector<int>& inst, std::vector<DavRun>& runs) {
  for (int k = 0; k < kMaxInst; ++k) B.h_tab->active[k] = 0;
  for (int i : inst) {
    B.h_tab->in[i] = runs[i].done ? nullptr : runs[i].px;
    B.h_tab->out[i] = runs[i].done ? nullptr : runs[i].py;
    B.h_tab->active[i] = runs[i].done ? 0 : 1;
  }
  for (int i : inst) {
    DMRG_CUDA(cudaEventRecord(B.ev_ctx[i], B.ctx[i]->stream));
    DMRG_CUDA(cudaStreamWaitEvent(B.bs, B.ev_ctx[i], 0));
  }
  DMRG_CUDA(cudaMemcpyAsync(B.d_tab, B.h_tab, sizeof(dmrg_batch::Tab), cudaMemcpyHostToDevice,
                            B.bs));
  DMRG_CUDA(cudaEventRecord(B.t0, B.bs));
  if (B.iter == 0) {
    batch_issue(B, inst);
  } else {
    if (!B.exec) {
      cudaGraph_t g = nullptr;
      DMRG_CUDA(cudaStreamBeginCapture(B.bs, cudaStreamCaptureModeThreadLocal));
      try {
        batch_issue(B, inst);
      } catch (...) {
        cudaStreamEndCapture(B.bs, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      DMRG_CUDA(cudaStreamEndCapture(B.bs, &g));
      cudaError_t e = cudaGraphInstantiate(&B.exec, g, 0);
      cudaGraphDestroy(g);
      DMRG_CUDA(e);
    }
    DMRG_CUDA(cudaGraphLaunch(B.exec, B.bs));
  }
  DMRG_CUDA(cudaEventRecord(B.t1, B.bs));
  DMRG_CUDA(cudaEventRecord(B.ev, B.bs));
  for (int i : inst) DMRG_CUDA(cudaStreamWaitEvent(B.ctx[i]->stream, B.ev, 0));
  DMRG_CUDA(cudaEventSynchronize(B.t1));
  float ms = 0;
  DMRG_CUDA(cudaEventElapsedTime(&ms, B.t0, B.t1));
  B.heff_seconds += ms * 1e-3;
  ++B.iter;
  ++B.products;
}

struct BWork {
  int inst, p, dir, M;
};

static void batch_step(dmrg_batch& B, const std::vector<BWork>& work,
                       std::vector<dmrg_step_stats>& st) {
  std::vector<int> inst;
  std::vector<DavRun> runs(B.ctx.size());
  std::vector<double> t0(B.ctx.size());
  // every instance's own bookkeeping (superblock, prediction, truncation, the host part of
  // its Davidson iterations) runs on its own host thread and its own stream
  WorkerPool& ip = WorkerPool::instances();
  ip.run(int(work.size()), [&](int j) {
    const BWork& w = work[j];
    Ctx& c = *B.ctx[w.inst];
    PoolScope ps(&c.pool);
    t0[w.inst] = now_s();
    Super& sb = super_at(c, w.p);
    c.psi_guess.alloc(std::max<int64_t>(sb.size, 1));
    predict(c, sb, w.p, w.dir, c.psi_guess.p);
    c.psi.alloc(std::max<int64_t>(sb.size, 1));
    dav_begin(c, sb, c.psi_guess.p, c.psi.p, runs[w.inst]);
  });
  for (const BWork& w : work) inst.push_back(w.inst);
  batch_buffers(B, inst);
  batch_lists(B, inst);
  if (B.exec) {
    cudaGraphExecDestroy(B.exec);
    B.exec = nullptr;
  }
  B.iter = 0;
  while (true) {
    bool any = false;
    for (int i : inst) any = any || !runs[i].done;
    if (!any) break;
    batch_product(B, inst, runs);
    ip.run(int(inst.size()), [&](int j) {
      const int i = inst[j];
      if (runs[i].done) return;
      PoolScope ps(&B.ctx[i]->pool);
      dav_after_product(*B.ctx[i], runs[i]);
    });
  }
  ip.run(int(work.size()), [&](int j) {
    const BWork& w = work[j];
    Ctx& c = *B.ctx[w.inst];
    PoolScope ps(&c.pool);
    c.psi_valid = true;
    c.psi_p = w.p;
    const double flops = c.sb->flops, bytes = c.sb->bytes;
    TruncResult tr = truncate_renormalize(c, w.p, w.dir, w.M);
    dav_energy(c, runs[w.inst].res);
    dmrg_step_stats& s = st[w.inst];
    s.p = w.p;
    s.dir = w.dir;
    s.n_products = runs[w.inst].res.nprod;
    s.kept = tr.kept;
    s.energy = runs[w.inst].res.theta;
    s.residual = runs[w.inst].res.resid;
    s.trunc_err = tr.trunc;
    s.seconds = now_s() - t0[w.inst];
    s.heff_seconds = 0;
    s.heff_flops = flops;
    s.heff_bytes = bytes;
    s.energy1 = NAN;
  });
}

}  // namespace dmrg

template <class F>
static int bguarded(dmrg_batch* b, F&& f) {
  if (!b) return DMRG_EINVAL;
  try {
    f();
    return DMRG_OK;
  } catch (const Error& e) {
    b->err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    b->err = "host allocation failed";
    return DMRG_ENOMEM;
  } catch (const std::exception& e) {
    b->err = e.what();
    return DMRG_EINVAL;
  }
}

extern "C" int dmrg_batch_create(int32_t n, dmrg_ctx* const* ctxs, dmrg_batch** out) {
  if (!out) return DMRG_EINVAL;
  *out = nullptr;
  dmrg_batch* b = nullptr;
  try {
    b = new dmrg_batch();
  } catch (...) {
    return DMRG_ENOMEM;
  }
  int rc = bguarded(b, [&] {
    DMRG_REQUIRE(n >= 1 && n <= kMaxInst && ctxs, DMRG_EINVAL, "batch size must be in [1, 64]");
    for (int i = 0; i < n; ++i) {
      DMRG_REQUIRE(ctxs[i] && ctxs[i]->N > 0, DMRG_EINVAL, "invalid context in batch");
      for (int j = 0; j < i; ++j)
        DMRG_REQUIRE(ctxs[i] != ctxs[j], DMRG_EINVAL, "a context appears twice in the batch");
      b->ctx.push_back(ctxs[i]);
    }
    b->precision = ctxs[0]->opt.precision;
    DMRG_CUDA(cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking));
    DMRG_CUDA(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
    b->ev_ctx.resize(n);
    for (int i = 0; i < n; ++i) DMRG_CUDA(cudaEventCreateWithFlags(&b->ev_ctx[i], cudaEventDisableTiming));
    DMRG_CUDA(cudaEventCreate(&b->t0));
    DMRG_CUDA(cudaEventCreate(&b->t1));
    DMRG_CUDA(cudaMallocHost(&b->h_tab, sizeof(dmrg_batch::Tab)));
    DMRG_CUDA(cudaMalloc(&b->d_tab, sizeof(dmrg_batch::Tab)));
  });
  *out = b;
  return rc;
}

extern "C" int dmrg_batch_destroy(dmrg_batch* b) {
  delete b;
  return DMRG_OK;
}

extern "C" const char* dmrg_batch_last_error(const dmrg_batch* b) {
  return b ? b->err.c_str() : "NULL batch";
}

extern "C" int dmrg_batch_sweep(dmrg_batch* b, const int32_t* M, double* energies,
                                dmrg_batch_stats* st) {
  return bguarded(b, [&] {
    DMRG_REQUIRE(M != nullptr, DMRG_EINVAL, "M is NULL");
    const int n = int(b->ctx.size());
    for (int i = 0; i < n; ++i) {
      DMRG_REQUIRE(b->ctx[i]->built, DMRG_EINVAL, "dmrg_build_blocks has not been called");
      DMRG_REQUIRE(b->ctx[i]->opt.precision == b->precision, DMRG_EINVAL,
                   "all contexts of a batch must use the same precision");
      DMRG_REQUIRE(M[i] >= 1, DMRG_EINVAL, "M must be positive");
      DMRG_REQUIRE(b->ctx[i]->n_roots == 1, DMRG_EINVAL,
                   "two-state targeting is not available in batch mode");
    }
    std::vector<std::vector<std::pair<int, int>>> seq(n);
    size_t len = 0;
    for (int i = 0; i < n; ++i) {
      const int N = b->ctx[i]->N;
      for (int p = 1; p <= N - 3; ++p) seq[i].push_back({p, 0});
      for (int p = N - 3; p >= 1; --p) seq[i].push_back({p, 1});
      len = std::max(len, seq[i].size());
    }
    const int64_t p0 = b->products;
    const double h0 = b->heff_seconds;
    const int64_t l0 = g_launches.load();
    std::vector<dmrg_step_stats> last(n), cur(n);
    for (size_t j = 0; j < len; ++j) {
      std::vector<BWork> work;
      for (int i = 0; i < n; ++i)
        if (j < seq[i].size()) work.push_back(BWork{i, seq[i][j].first, seq[i][j].second, M[i]});
      batch_step(*b, work, cur);
      for (const BWork& w : work) last[w.inst] = cur[w.inst];
    }
    if (energies)
      for (int i = 0; i < n; ++i) energies[i] = last[i].energy;
    if (st) {
      st->products = b->products - p0;
      st->heff_seconds = b->heff_seconds - h0;
      st->launches = g_launches.load() - l0;
    }
  });
}
