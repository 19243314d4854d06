// Host-side problem bookkeeping: chain-ordered Hamiltonian and the normal/complementary
// operator partition (a matrix-product operator) used by every two-site step.
#pragma once
#include "common.h"

namespace dmrg {

enum LabT : int8_t { L_I = 0, L_H, L_CD, L_C, L_S, L_SD, L_A, L_AD, L_B, L_P, L_PD, L_Q };
struct Label {
  int8_t t;
  int16_t i, j;
};
enum SiteOp : int8_t { OP_I = 0, OP_N = 1, OP_CD = 2, OP_C = 3 };

// W[s] entry: left_b(bond s) += left_a(bond s-1) . op_s  (and right_a += op . right_b)
struct WEntry {
  int32_t a, b;
  int8_t op;
  double coef;
};

struct Chain {
  int N = 0;
  std::vector<QN> q;          // site quantum numbers in chain order
  std::vector<double> eps;    // chain order
  std::vector<double> W4;     // antisymmetrised two-body tensor over chain positions
  QN target{0, 0, 0};
  double W(int i, int j, int k, int l) const {
    return W4[((size_t(i) * N + j) * N + k) * N + l];
  }
};

struct MPO {
  int N = 0;
  std::vector<std::vector<Label>> labels;    // index b+1 for bond b = -1..N-1
  std::vector<std::vector<int8_t>> parity;   // fermion parity of each label
  std::vector<std::vector<QN>> dq;           // quantum-number change of the left operator
  std::vector<std::vector<WEntry>> W;        // per site s = 0..N-1
};

void build_chain(const dmrg_problem* p, Chain& c);
void build_mpo(const Chain& c, MPO& m);

}  // namespace dmrg
