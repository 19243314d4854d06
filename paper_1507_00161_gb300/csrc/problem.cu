// Chain-ordered Hamiltonian (Eq. 1) and its partition into block-operator products.
//
// Bond b separates left sites {0..b} from right sites {b+1..N-1}.  With the
// antisymmetrised W (two-body part 1/4 sum W_ijkl c+_i c+_j c_l c_k) every term of H
// is a product (left operator)(right operator), fermionic order left first:
//   H^L 1 + 1 H^R
//   + sum_{i in L} c+_i S^R_i - c_i (S^R_i)^+   + sum_{j in R} S^L_j c+_j - (S^L_j)^+ c_j
//   + pair terms with normal operators A_ij = c+_i c+_j, A_ij^+, B_ik = c+_i c_k on the
//     side with fewer sites and complementary ones P_kl = sum W_ijkl c+_i c+_j,
//     Q_jl = sum W_ijkl c+_i c_k on the other,
// S^L_j = 1/2 sum_{ikl in L} W_ijkl c+_i c_l c_k.  Growing the left block by one site gives
// a linear recursion (left_b(s) = sum_a left_a(s-1) . op_s), i.e. a matrix-product
// operator; the right blocks use the same entries.  Labels unreachable from the vacuum
// identity or not leading to the final H are dropped.
#include <unordered_map>
#include <unordered_set>

#include "problem.h"

namespace dmrg {

void build_chain(const dmrg_problem* p, Chain& c) {
  DMRG_REQUIRE(p != nullptr, DMRG_EINVAL, "problem is NULL");
  const int N = p->n_sites;
  DMRG_REQUIRE(N >= 4 && N <= 64, DMRG_EINVAL, "n_sites must be in [4, 64]");
  DMRG_REQUIRE(p->species && p->two_m && p->eps && p->order, DMRG_EINVAL, "NULL site array");
  DMRG_REQUIRE(p->n_v >= 0 && (p->n_v == 0 || (p->v_idx && p->v_val)), DMRG_EINVAL,
               "bad two-body list");
  std::vector<int> pos(N, -1);
  for (int cpos = 0; cpos < N; ++cpos) {
    int s = p->order[cpos];
    DMRG_REQUIRE(s >= 0 && s < N && pos[s] < 0, DMRG_EINVAL, "order is not a permutation");
    pos[s] = cpos;
  }
  c.N = N;
  c.q.resize(N);
  c.eps.resize(N);
  std::vector<QN> qsite(N);
  for (int s = 0; s < N; ++s) {
    DMRG_REQUIRE(p->species[s] == 0 || p->species[s] == 1, DMRG_EINVAL, "species must be 0/1");
    qsite[s] = p->species[s] == 0 ? QN{1, 0, p->two_m[s]} : QN{0, 1, p->two_m[s]};
  }
  for (int cpos = 0; cpos < N; ++cpos) {
    c.q[cpos] = qsite[p->order[cpos]];
    c.eps[cpos] = p->eps[p->order[cpos]];
  }
  c.target = QN{p->Np, p->Nn, p->two_Mz};
  c.W4.assign(size_t(N) * N * N * N, 0.0);
  // canonical list in chain positions, then antisymmetrise
  std::vector<double> vb(size_t(N) * N * N * N, 0.0);
  for (int64_t t = 0; t < p->n_v; ++t) {
    int i = p->v_idx[4 * t], j = p->v_idx[4 * t + 1], k = p->v_idx[4 * t + 2],
        l = p->v_idx[4 * t + 3];
    DMRG_REQUIRE(i >= 0 && j < N && k >= 0 && l < N && i < j && k < l, DMRG_EINVAL,
                 "two-body index out of range or not i<j, k<l");
    DMRG_REQUIRE(qsite[i] + qsite[j] == qsite[k] + qsite[l], DMRG_EINVAL,
                 "two-body entry does not conserve (N_p, N_n, 2M)");
    int ci = pos[i], cj = pos[j], ck = pos[k], cl = pos[l];
    double sg = 1.0;
    if (ci > cj) { std::swap(ci, cj); sg = -sg; }
    if (ck > cl) { std::swap(ck, cl); sg = -sg; }
    vb[((size_t(ci) * N + cj) * N + ck) * N + cl] += sg * p->v_val[t];
  }
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j)
      for (int k = 0; k < N; ++k)
        for (int l = k + 1; l < N; ++l) {
          double v = vb[((size_t(i) * N + j) * N + k) * N + l];
          double w = vb[((size_t(k) * N + l) * N + i) * N + j];
          DMRG_REQUIRE(v == w, DMRG_EINVAL, "two-body list is not Hermitian");
          if (v == 0.0) continue;
          auto at = [&](int a, int b, int cc, int d) -> double& {
            return c.W4[((size_t(a) * N + b) * N + cc) * N + d];
          };
          at(i, j, k, l) = v;
          at(j, i, k, l) = -v;
          at(i, j, l, k) = -v;
          at(j, i, l, k) = v;
        }
}

static inline int64_t key_of(int t, int i, int j) {
  return (int64_t(t) << 20) | (int64_t(i + 1) << 10) | int64_t(j + 1);
}

static bool normal_mode(int b, int N) { return (b + 1) <= (N - b - 1); }

static std::vector<Label> raw_labels(int b, int N) {
  std::vector<Label> out;
  auto push = [&](int t, int i, int j) { out.push_back(Label{int8_t(t), int16_t(i), int16_t(j)}); };
  push(L_I, -1, -1);
  push(L_H, -1, -1);
  for (int i = 0; i <= b; ++i) push(L_CD, i, -1);
  for (int i = 0; i <= b; ++i) push(L_C, i, -1);
  for (int j = b + 1; j < N; ++j) push(L_S, j, -1);
  for (int j = b + 1; j < N; ++j) push(L_SD, j, -1);
  if (normal_mode(b, N)) {
    for (int i = 0; i <= b; ++i)
      for (int j = i + 1; j <= b; ++j) push(L_A, i, j);
    for (int i = 0; i <= b; ++i)
      for (int j = i + 1; j <= b; ++j) push(L_AD, i, j);
    for (int i = 0; i <= b; ++i)
      for (int k = 0; k <= b; ++k) push(L_B, i, k);
  } else {
    for (int k = b + 1; k < N; ++k)
      for (int l = k + 1; l < N; ++l) push(L_P, k, l);
    for (int k = b + 1; k < N; ++k)
      for (int l = k + 1; l < N; ++l) push(L_PD, k, l);
    for (int j = b + 1; j < N; ++j)
      for (int l = b + 1; l < N; ++l) push(L_Q, j, l);
  }
  return out;
}

static int label_parity(const Label& l) {
  return (l.t == L_CD || l.t == L_C || l.t == L_S || l.t == L_SD) ? 1 : 0;
}

static QN label_dq(const Label& l, const std::vector<QN>& q) {
  QN z{0, 0, 0};
  switch (l.t) {
    case L_I:
    case L_H: return z;
    case L_CD: return q[l.i];
    case L_C: return z - q[l.i];
    case L_S: return z - q[l.i];
    case L_SD: return q[l.i];
    case L_A: return q[l.i] + q[l.j];
    case L_AD: return z - (q[l.i] + q[l.j]);
    case L_B: return q[l.i] - q[l.j];
    case L_P: return q[l.i] + q[l.j];
    case L_PD: return z - (q[l.i] + q[l.j]);
    case L_Q: return q[l.j] - q[l.i];
  }
  return z;
}

struct RawEntry {
  int64_t a;   // key at bond s-1
  int32_t b;   // raw index at bond s
  int8_t op;
  double coef;
};

// entries of W[s] on raw labels (see the recursion in the file comment)
static void site_entries(int s, const Chain& c, const std::unordered_map<int64_t, int>& prev,
                         const std::vector<Label>& cur, std::vector<RawEntry>& E) {
  const int N = c.N;
  const bool mprev = normal_mode(s - 1, N);
  auto W = [&](int i, int j, int k, int l) { return c.W(i, j, k, l); };
  auto add = [&](int t, int i, int j, int b, int op, double coef) {
    if (coef == 0.0) return;
    int64_t k = key_of(t, i, j);
    if (prev.find(k) == prev.end()) return;
    E.push_back(RawEntry{k, b, int8_t(op), coef});
  };
  for (int b = 0; b < int(cur.size()); ++b) {
    const Label& lab = cur[b];
    switch (lab.t) {
      case L_I: add(L_I, -1, -1, b, OP_I, 1.0); break;
      case L_H:
        add(L_H, -1, -1, b, OP_I, 1.0);
        add(L_I, -1, -1, b, OP_N, c.eps[s]);
        add(L_S, s, -1, b, OP_CD, 1.0);
        add(L_SD, s, -1, b, OP_C, -1.0);
        if (mprev) {
          for (int i = 0; i < s; ++i)
            for (int k = 0; k < s; ++k) add(L_B, i, k, b, OP_N, W(i, s, k, s));
        } else {
          add(L_Q, s, s, b, OP_N, 1.0);
        }
        break;
      case L_CD:
      case L_C:
        if (lab.i < s) add(lab.t, lab.i, -1, b, OP_I, 1.0);
        else add(L_I, -1, -1, b, lab.t == L_CD ? OP_CD : OP_C, 1.0);
        break;
      case L_S: {
        int j = lab.i;
        add(L_S, j, -1, b, OP_I, 1.0);
        if (mprev) {
          for (int k = 0; k < s; ++k)
            for (int l = k + 1; l < s; ++l) add(L_AD, k, l, b, OP_CD, W(s, j, k, l));
          for (int i = 0; i < s; ++i)
            for (int k = 0; k < s; ++k) add(L_B, i, k, b, OP_C, -W(i, j, k, s));
        } else {
          add(L_PD, s, j, b, OP_CD, 1.0);
          add(L_Q, j, s, b, OP_C, -1.0);
        }
        for (int k = 0; k < s; ++k) add(L_C, k, -1, b, OP_N, W(s, j, k, s));
        break;
      }
      case L_SD: {
        int j = lab.i;
        add(L_SD, j, -1, b, OP_I, 1.0);
        if (mprev) {
          for (int k = 0; k < s; ++k)
            for (int l = k + 1; l < s; ++l) add(L_A, k, l, b, OP_C, W(s, j, k, l));
          for (int x = 0; x < s; ++x)
            for (int y = 0; y < s; ++y) add(L_B, x, y, b, OP_CD, -W(y, j, x, s));
        } else {
          add(L_P, s, j, b, OP_C, 1.0);
          add(L_Q, s, j, b, OP_CD, -1.0);
        }
        for (int k = 0; k < s; ++k) add(L_CD, k, -1, b, OP_N, W(s, j, k, s));
        break;
      }
      case L_A:
      case L_AD:
        if (lab.j < s) add(lab.t, lab.i, lab.j, b, OP_I, 1.0);
        else if (lab.t == L_A) add(L_CD, lab.i, -1, b, OP_CD, 1.0);
        else add(L_C, lab.i, -1, b, OP_C, -1.0);
        break;
      case L_B: {
        int i = lab.i, k = lab.j;
        if (i < s && k < s) add(L_B, i, k, b, OP_I, 1.0);
        else if (i == s && k < s) add(L_C, k, -1, b, OP_CD, -1.0);
        else if (k == s && i < s) add(L_CD, i, -1, b, OP_C, 1.0);
        else add(L_I, -1, -1, b, OP_N, 1.0);
        break;
      }
      case L_P:
      case L_PD: {
        int k = lab.i, l = lab.j;
        if (mprev) {
          int src = lab.t == L_P ? L_A : L_AD;
          for (int i = 0; i < s; ++i)
            for (int j = i + 1; j < s; ++j) add(src, i, j, b, OP_I, W(i, j, k, l));
        } else {
          add(lab.t, k, l, b, OP_I, 1.0);
        }
        for (int i = 0; i < s; ++i) {
          if (lab.t == L_P) add(L_CD, i, -1, b, OP_CD, W(i, s, k, l));
          else add(L_C, i, -1, b, OP_C, -W(i, s, k, l));
        }
        break;
      }
      case L_Q: {
        int j = lab.i, l = lab.j;
        if (mprev) {
          for (int i = 0; i < s; ++i)
            for (int k = 0; k < s; ++k) add(L_B, i, k, b, OP_I, W(i, j, k, l));
        } else {
          add(L_Q, j, l, b, OP_I, 1.0);
        }
        for (int k = 0; k < s; ++k) add(L_C, k, -1, b, OP_CD, -W(s, j, k, l));
        for (int i = 0; i < s; ++i) add(L_CD, i, -1, b, OP_C, W(i, j, s, l));
        add(L_I, -1, -1, b, OP_N, W(s, j, s, l));
        break;
      }
    }
  }
}

void build_mpo(const Chain& c, MPO& m) {
  const int N = c.N;
  m.N = N;
  std::vector<std::vector<Label>> raw(N + 1);
  raw[0] = {Label{L_I, -1, -1}};
  for (int b = 0; b < N - 1; ++b) raw[b + 1] = raw_labels(b, N);
  raw[N] = {Label{L_H, -1, -1}};
  std::vector<std::unordered_map<int64_t, int>> rawidx(N + 1);
  for (int x = 0; x <= N; ++x)
    for (int k = 0; k < int(raw[x].size()); ++k)
      rawidx[x][key_of(raw[x][k].t, raw[x][k].i, raw[x][k].j)] = k;
  std::vector<std::vector<RawEntry>> E(N);
  for (int s = 0; s < N; ++s) site_entries(s, c, rawidx[s], raw[s + 1], E[s]);
  // reachability
  std::vector<std::vector<char>> fw(N + 1), bw(N + 1);
  for (int x = 0; x <= N; ++x) {
    fw[x].assign(raw[x].size(), 0);
    bw[x].assign(raw[x].size(), 0);
  }
  fw[0][0] = 1;
  for (int s = 0; s < N; ++s)
    for (auto& e : E[s])
      if (fw[s][rawidx[s].at(e.a)]) fw[s + 1][e.b] = 1;
  bw[N][0] = 1;
  for (int s = N - 1; s >= 0; --s)
    for (auto& e : E[s])
      if (bw[s + 1][e.b]) bw[s][rawidx[s].at(e.a)] = 1;
  std::vector<std::vector<int>> newidx(N + 1);
  m.labels.assign(N + 1, {});
  m.parity.assign(N + 1, {});
  m.dq.assign(N + 1, {});
  for (int x = 0; x <= N; ++x) {
    newidx[x].assign(raw[x].size(), -1);
    for (int k = 0; k < int(raw[x].size()); ++k)
      if (fw[x][k] && bw[x][k]) {
        newidx[x][k] = int(m.labels[x].size());
        m.labels[x].push_back(raw[x][k]);
        m.parity[x].push_back(int8_t(label_parity(raw[x][k])));
        m.dq[x].push_back(label_dq(raw[x][k], c.q));
      }
  }
  m.W.assign(N, {});
  for (int s = 0; s < N; ++s) {
    for (auto& e : E[s]) {
      int a = newidx[s][rawidx[s].at(e.a)], b = newidx[s + 1][e.b];
      if (a < 0 || b < 0) continue;
      m.W[s].push_back(WEntry{a, b, e.op, e.coef});
      // consistency of quantum numbers and parity
      QN dop = e.op == OP_CD ? c.q[s] : (e.op == OP_C ? QN{0, 0, 0} - c.q[s] : QN{0, 0, 0});
      DMRG_REQUIRE(m.dq[s][a] + dop == m.dq[s + 1][b], DMRG_EINVAL,
                   "internal: operator partition violates quantum numbers");
      int pop = (e.op == OP_CD || e.op == OP_C) ? 1 : 0;
      DMRG_REQUIRE(((m.parity[s][a] + pop) & 1) == m.parity[s + 1][b], DMRG_EINVAL,
                   "internal: operator partition violates fermion parity");
    }
  }
}

}  // namespace dmrg
