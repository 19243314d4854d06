/*
 * Oracle: the exact lowest eigenpair of the shell-model Hamiltonian of Eq. (1) in one
 * m-scheme sector, by the Lanczos method with full reorthogonalisation, in FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  Called through ctypes from oracle/hamiltonian.py (tests,
 * the scripts that write stored expected values); the CUDA library never links or calls
 * it, and it shares no code with it.
 *
 * What it computes (the plain definition, no factorisation tricks):
 *   H = sum_i eps_i n_i + sum_{i<j, k<l} vbar[ij,kl] c+_i c+_j c_l c_k      (Eq. 1)
 * on Slater determinants |s> = c+_{a_1} c+_{a_2} ... c+_{a_n} |0>, a_1 < a_2 < ... site
 * indices, with c_x |s> = (-1)^{#(occupied sites below x)} |s \ x> and the same sign for
 * c+_x.  The basis of the sector (N_p, N_n, 2M) is every determinant with N_p proton and
 * N_n neutron sites occupied and sum of 2m = 2M, ordered by the 2M of its protons, then
 * its proton configuration, then its neutron configuration (the order only fixes the
 * vector layout).
 *
 * y = H x is formed row by row: applying every term of H to the determinant s gives the
 * column <t|H|s>; because the two-body list is Hermitian (both (ij,kl) and (kl,ij), equal
 * values: the caller checks this) H is real symmetric and <s|H|t> = <t|H|s>, so
 *   y[s] = sum_t <t|H|s> x[t].
 * Rows are split over threads; each row is written by one thread only.
 *
 * Lanczos (the textbook three-term recursion): v_1 = a fixed start vector, normalised;
 *   w = H v_j - beta_{j-1} v_{j-1},  alpha_j = <v_j, w>,  w -= alpha_j v_j,
 * then w is orthogonalised twice against every v_1..v_j (classical Gram-Schmidt, full
 * reorthogonalisation), beta_j = |w|, v_{j+1} = w / beta_j.  After each step the lowest
 * eigenvalue theta of the tridiagonal T_j is found by bisection with Sturm counts and its
 * eigenvector y by inverse iteration; the Ritz pair's residual norm is beta_j |y_j|.  Stop
 * when that residual is <= tol and theta moved by less than 1e-13 (1 + |theta|) since the
 * previous step, or at max_iter.  The Ritz vector x = sum_j y_j v_j is returned with its
 * residual |H x - theta x| recomputed explicitly.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------------- */
/* configurations of one species: all choices of n sites among that species' sites    */
/* ---------------------------------------------------------------------------------- */
typedef struct {
  int n_conf;
  uint64_t* mask;     /* [n_conf] full site masks, grouped by 2M, ascending mask inside */
  int* two_m;         /* [n_conf] total 2m of the configuration                        */
  int* rank;          /* [n_conf] position inside its 2M group                         */
  int* group;         /* [n_conf] its 2M group                                         */
  int n_groups;
  int* g_two_m;       /* [n_groups] 2M of each group, ascending                          */
  int* g_start;       /* [n_groups + 1] configuration ranges                              */
  /* open-addressing table mask -> configuration index */
  uint64_t* h_key;
  int* h_val;
  uint64_t h_mask;
} Species;

static uint64_t mix64(uint64_t x) {
  x *= 0x9E3779B97F4A7C15ULL;   /* Fibonacci hashing: the table size is a power of two */
  return x ^ (x >> 29);
}

static int species_lookup(const Species* sp, uint64_t key) {
  uint64_t h = mix64(key) & sp->h_mask;
  while (sp->h_val[h] >= 0) {
    if (sp->h_key[h] == key) return sp->h_val[h];
    h = (h + 1) & sp->h_mask;
  }
  return -1;
}

static void species_free(Species* sp) {
  free(sp->mask);
  free(sp->two_m);
  free(sp->rank);
  free(sp->group);
  free(sp->g_two_m);
  free(sp->g_start);
  free(sp->h_key);
  free(sp->h_val);
  memset(sp, 0, sizeof(*sp));
}

typedef struct {
  uint64_t mask;
  int two_m;
} Conf;

static int conf_cmp(const void* a, const void* b) {
  const Conf* x = (const Conf*)a;
  const Conf* y = (const Conf*)b;
  if (x->two_m != y->two_m) return x->two_m < y->two_m ? -1 : 1;
  if (x->mask != y->mask) return x->mask < y->mask ? -1 : 1;
  return 0;
}

/* every n-subset of the sites in `sites` (count ns) */
static int species_build(Species* sp, const int* sites, const int* tm, int ns, int n) {
  memset(sp, 0, sizeof(*sp));
  if (n < 0 || n > ns) return -1;
  /* number of subsets: binomial(ns, n) */
  double cnt = 1.0;
  for (int i = 0; i < n; ++i) cnt = cnt * (ns - i) / (i + 1);
  if (cnt > 5e7) return -1;
  const int nc = (int)(cnt + 0.5);
  Conf* c = (Conf*)malloc(sizeof(Conf) * (size_t)(nc > 0 ? nc : 1));
  int* pick = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) pick[i] = i;
  int k = 0;
  for (;;) {
    uint64_t m = 0;
    int t = 0;
    for (int i = 0; i < n; ++i) {
      m |= 1ULL << sites[pick[i]];
      t += tm[pick[i]];
    }
    c[k].mask = m;
    c[k].two_m = t;
    ++k;
    /* next combination in lexicographic order */
    int i = n - 1;
    while (i >= 0 && pick[i] == ns - n + i) --i;
    if (i < 0) break;
    ++pick[i];
    for (int j = i + 1; j < n; ++j) pick[j] = pick[j - 1] + 1;
  }
  free(pick);
  qsort(c, (size_t)nc, sizeof(Conf), conf_cmp);
  sp->n_conf = nc;
  sp->mask = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)nc);
  sp->two_m = (int*)malloc(sizeof(int) * (size_t)nc);
  sp->rank = (int*)malloc(sizeof(int) * (size_t)nc);
  sp->group = (int*)malloc(sizeof(int) * (size_t)nc);
  sp->g_two_m = (int*)malloc(sizeof(int) * (size_t)(nc + 1));
  sp->g_start = (int*)malloc(sizeof(int) * (size_t)(nc + 2));
  int g = -1;
  for (int i = 0; i < nc; ++i) {
    sp->mask[i] = c[i].mask;
    sp->two_m[i] = c[i].two_m;
    if (i == 0 || c[i].two_m != c[i - 1].two_m) {
      ++g;
      sp->g_two_m[g] = c[i].two_m;
      sp->g_start[g] = i;
    }
    sp->rank[i] = i - sp->g_start[g];
    sp->group[i] = g;
  }
  sp->n_groups = g + 1;
  sp->g_start[sp->n_groups] = nc;
  free(c);
  uint64_t cap = 16;
  while (cap < 2 * (uint64_t)nc) cap <<= 1;
  sp->h_mask = cap - 1;
  sp->h_key = (uint64_t*)malloc(sizeof(uint64_t) * cap);
  sp->h_val = (int*)malloc(sizeof(int) * cap);
  for (uint64_t i = 0; i < cap; ++i) sp->h_val[i] = -1;
  for (int i = 0; i < nc; ++i) {
    uint64_t h = mix64(sp->mask[i]) & sp->h_mask;
    while (sp->h_val[h] >= 0) h = (h + 1) & sp->h_mask;
    sp->h_key[h] = sp->mask[i];
    sp->h_val[h] = i;
  }
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* the sector basis and H                                                              */
/* ---------------------------------------------------------------------------------- */
typedef struct {
  int N;
  double eps[64];
  uint64_t pmask_all, nmask_all;
  Species P, Nn;
  int two_M;
  /* blocks: proton 2M group gp with neutron group gn, 2M_p + 2M_n = 2M */
  int n_blocks;
  int* b_gp;
  int* b_gn;
  int64_t* b_base;    /* [n_blocks + 1] */
  int* gp_block;      /* proton group -> block (or -1) */
  int64_t* p_base;    /* proton configuration -> b_base + rank * (block's neutron count), or -1 */
  int* n_group;       /* neutron configuration -> its group (== the block's gn when valid) */
  int64_t dim;
  /* two-body list in CSR by annihilated pair (k, l), k < l: pair index k * N + l */
  int64_t* pair_ptr;  /* [N*N + 1] */
  int* ti;
  int* tj;
  double* tv;
} Sector;

static void sector_free(Sector* S) {
  species_free(&S->P);
  species_free(&S->Nn);
  free(S->b_gp);
  free(S->b_gn);
  free(S->b_base);
  free(S->gp_block);
  free(S->p_base);
  free(S->pair_ptr);
  free(S->ti);
  free(S->tj);
  free(S->tv);
  memset(S, 0, sizeof(*S));
}

static int sector_build(Sector* S, int N, const int8_t* species, const int8_t* two_m,
                        const double* eps, int64_t n_v, const int32_t* v_idx,
                        const double* v_val, int Np, int Nn, int two_M) {
  memset(S, 0, sizeof(*S));
  if (N < 1 || N > 64) return -1;
  S->N = N;
  S->two_M = two_M;
  int ps[64], pm[64], nsit[64], nm[64], np_ = 0, nn_ = 0;
  for (int i = 0; i < N; ++i) {
    S->eps[i] = eps[i];
    if (species[i] == 0) {
      ps[np_] = i;
      pm[np_++] = two_m[i];
      S->pmask_all |= 1ULL << i;
    } else {
      nsit[nn_] = i;
      nm[nn_++] = two_m[i];
      S->nmask_all |= 1ULL << i;
    }
  }
  if (species_build(&S->P, ps, pm, np_, Np) != 0) return -1;
  if (species_build(&S->Nn, nsit, nm, nn_, Nn) != 0) return -1;
  S->b_gp = (int*)malloc(sizeof(int) * (size_t)(S->P.n_groups + 1));
  S->b_gn = (int*)malloc(sizeof(int) * (size_t)(S->P.n_groups + 1));
  S->b_base = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->P.n_groups + 2));
  S->gp_block = (int*)malloc(sizeof(int) * (size_t)(S->P.n_groups + 1));
  int64_t base = 0;
  S->n_blocks = 0;
  for (int gp = 0; gp < S->P.n_groups; ++gp) {
    S->gp_block[gp] = -1;
    const int want = two_M - S->P.g_two_m[gp];
    for (int gn = 0; gn < S->Nn.n_groups; ++gn)
      if (S->Nn.g_two_m[gn] == want) {
        const int b = S->n_blocks++;
        S->b_gp[b] = gp;
        S->b_gn[b] = gn;
        S->b_base[b] = base;
        S->gp_block[gp] = b;
        base += (int64_t)(S->P.g_start[gp + 1] - S->P.g_start[gp]) *
                (S->Nn.g_start[gn + 1] - S->Nn.g_start[gn]);
      }
  }
  S->b_base[S->n_blocks] = base;
  S->dim = base;
  S->p_base = (int64_t*)malloc(sizeof(int64_t) * (size_t)S->P.n_conf);
  for (int ip = 0; ip < S->P.n_conf; ++ip) {
    const int b = S->gp_block[S->P.group[ip]];
    if (b < 0) {
      S->p_base[ip] = -1;
      continue;
    }
    const int gn = S->b_gn[b];
    S->p_base[ip] = S->b_base[b] + (int64_t)S->P.rank[ip] * (S->Nn.g_start[gn + 1] - S->Nn.g_start[gn]);
  }
  S->n_group = S->Nn.group;
  /* two-body terms grouped by the annihilated pair */
  const int64_t npair = (int64_t)N * N;
  S->pair_ptr = (int64_t*)calloc((size_t)(npair + 1), sizeof(int64_t));
  for (int64_t t = 0; t < n_v; ++t) {
    const int i = v_idx[4 * t], j = v_idx[4 * t + 1], k = v_idx[4 * t + 2], l = v_idx[4 * t + 3];
    if (i < 0 || j < 0 || k < 0 || l < 0 || i >= N || j >= N || k >= N || l >= N || !(i < j) ||
        !(k < l))
      return -2;
    S->pair_ptr[(int64_t)k * N + l + 1] += 1;
  }
  for (int64_t p = 0; p < npair; ++p) S->pair_ptr[p + 1] += S->pair_ptr[p];
  S->ti = (int*)malloc(sizeof(int) * (size_t)(n_v > 0 ? n_v : 1));
  S->tj = (int*)malloc(sizeof(int) * (size_t)(n_v > 0 ? n_v : 1));
  S->tv = (double*)malloc(sizeof(double) * (size_t)(n_v > 0 ? n_v : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)npair);
  memcpy(fill, S->pair_ptr, sizeof(int64_t) * (size_t)npair);
  for (int64_t t = 0; t < n_v; ++t) {
    const int i = v_idx[4 * t], j = v_idx[4 * t + 1], k = v_idx[4 * t + 2], l = v_idx[4 * t + 3];
    const int64_t pos = fill[(int64_t)k * N + l]++;
    S->ti[pos] = i;
    S->tj[pos] = j;
    S->tv[pos] = v_val[t];
  }
  free(fill);
  return 0;
}

/* basis index of a determinant mask, -1 if outside the sector */
static int64_t sector_index(const Sector* S, uint64_t s) {
  const int ip = species_lookup(&S->P, s & S->pmask_all);
  const int in = species_lookup(&S->Nn, s & S->nmask_all);
  if (ip < 0 || in < 0) return -1;
  const int64_t pb = S->p_base[ip];
  if (pb < 0) return -1;
  if (S->n_group[in] != S->b_gn[S->gp_block[S->P.group[ip]]]) return -1;
  return pb + S->Nn.rank[in];
}

/* determinant mask of basis index r */
static uint64_t sector_mask(const Sector* S, int64_t r) {
  int b = 0;
  while (S->b_base[b + 1] <= r) ++b;
  const int gp = S->b_gp[b], gn = S->b_gn[b];
  const int dn = S->Nn.g_start[gn + 1] - S->Nn.g_start[gn];
  const int64_t q = r - S->b_base[b];
  const int ip = S->P.g_start[gp] + (int)(q / dn);
  const int in = S->Nn.g_start[gn] + (int)(q % dn);
  return S->P.mask[ip] | S->Nn.mask[in];
}

static int parity_below(uint64_t s, int x) {
  return __builtin_popcountll(s & ((1ULL << x) - 1ULL)) & 1;
}

/* y[r] for rows r in [r0, r1): y[s] = sum_t <t|H|s> x[t] */
static void apply_rows(const Sector* S, const double* x, double* y, int64_t r0, int64_t r1) {
  const int N = S->N;
  int occ[64];
  for (int64_t r = r0; r < r1; ++r) {
    const uint64_t s = sector_mask(S, r);
    int n = 0;
    double d = 0.0;
    for (int a = 0; a < N; ++a)
      if ((s >> a) & 1ULL) {
        occ[n++] = a;
        d += S->eps[a];
      }
    double acc = d * x[r];
    for (int a = 0; a < n; ++a)
      for (int b = a + 1; b < n; ++b) {
        const int k = occ[a], l = occ[b];
        const int64_t p0 = S->pair_ptr[(int64_t)k * N + l], p1 = S->pair_ptr[(int64_t)k * N + l + 1];
        /* c+_i c+_j c_l c_k |s>: c_k then c_l act first, the same for every (i, j) */
        const int sgkl = parity_below(s, k) ^ parity_below(s ^ (1ULL << k), l);
        const uint64_t base = s ^ (1ULL << k) ^ (1ULL << l);
        for (int64_t t = p0; t < p1; ++t) {
          const int i = S->ti[t], j = S->tj[t];
          if (base & ((1ULL << i) | (1ULL << j))) continue;   /* i or j already occupied */
          uint64_t u = base | (1ULL << j);
          const int sg = sgkl ^ parity_below(base, j) ^ parity_below(u, i);
          u |= 1ULL << i;
          const int64_t c = sector_index(S, u);
          if (c < 0) continue;   /* cannot happen for terms that conserve N_p, N_n, 2M */
          acc += (sg ? -S->tv[t] : S->tv[t]) * x[c];
        }
      }
    y[r] = acc;
  }
}

typedef struct {
  const Sector* S;
  const double* x;
  double* y;
  int64_t r0, r1;
} ApplyJob;

static void* apply_thread(void* arg) {
  ApplyJob* j = (ApplyJob*)arg;
  apply_rows(j->S, j->x, j->y, j->r0, j->r1);
  return NULL;
}

static void apply_h(const Sector* S, const double* x, double* y, int nt) {
  if (nt < 1) nt = 1;
  if (nt > 256) nt = 256;
  pthread_t th[256];
  ApplyJob jobs[256];
  for (int t = 0; t < nt; ++t) {
    jobs[t].S = S;
    jobs[t].x = x;
    jobs[t].y = y;
    jobs[t].r0 = S->dim * t / nt;
    jobs[t].r1 = S->dim * (t + 1) / nt;
  }
  for (int t = 1; t < nt; ++t) pthread_create(&th[t], NULL, apply_thread, &jobs[t]);
  apply_thread(&jobs[0]);
  for (int t = 1; t < nt; ++t) pthread_join(th[t], NULL);
}

/* ---------------------------------------------------------------------------------- */
/* symmetric tridiagonal T (diagonal a[0..m), off-diagonal b[0..m-1)): lowest          */
/* eigenvalue by bisection, eigenvector by inverse iteration                           */
/* ---------------------------------------------------------------------------------- */
/* number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots) */
static int sturm_count(const double* a, const double* b, int m, double x) {
  int c = 0;
  double q = a[0] - x;
  if (q < 0.0) ++c;
  for (int i = 1; i < m; ++i) {
    const double qq = (q == 0.0) ? 1e-300 : q;
    q = a[i] - x - b[i - 1] * b[i - 1] / qq;
    if (q < 0.0) ++c;
  }
  return c;
}

static double tri_lowest(const double* a, const double* b, int m) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
    if (a[i] - r < lo) lo = a[i] - r;
    if (a[i] + r > hi) hi = a[i] + r;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, m, mid) >= 1) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* solve (T - s I) z = y in place (Gaussian elimination with partial pivoting on the band) */
static void tri_solve(const double* a, const double* b, int m, double s, double* y) {
  double* d = (double*)malloc(sizeof(double) * (size_t)m);   /* diagonal of U   */
  double* e = (double*)malloc(sizeof(double) * (size_t)m);   /* first super     */
  double* f = (double*)malloc(sizeof(double) * (size_t)m);   /* second super    */
  double* sub = (double*)malloc(sizeof(double) * (size_t)m); /* current subdiag */
  for (int i = 0; i < m; ++i) {
    d[i] = a[i] - s;
    e[i] = i + 1 < m ? b[i] : 0.0;
    f[i] = 0.0;
    sub[i] = i + 1 < m ? b[i] : 0.0;
  }
  for (int i = 0; i + 1 < m; ++i) {
    /* rows i and i+1: [d_i e_i f_i ; sub_i d_{i+1} e_{i+1}] */
    if (fabs(sub[i]) > fabs(d[i])) {
      double t;
      t = d[i]; d[i] = sub[i]; sub[i] = t;
      t = e[i]; e[i] = d[i + 1]; d[i + 1] = t;
      t = f[i]; f[i] = e[i + 1]; e[i + 1] = t;
      t = y[i]; y[i] = y[i + 1]; y[i + 1] = t;
    }
    const double piv = d[i] == 0.0 ? 1e-300 : d[i];
    const double l = sub[i] / piv;
    d[i + 1] -= l * e[i];
    e[i + 1] -= l * f[i];
    y[i + 1] -= l * y[i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double v = y[i];
    if (i + 1 < m) v -= e[i] * y[i + 1];
    if (i + 2 < m) v -= f[i] * y[i + 2];
    const double piv = d[i] == 0.0 ? 1e-300 : d[i];
    y[i] = v / piv;
  }
  free(d);
  free(e);
  free(f);
  free(sub);
}

static void tri_vector(const double* a, const double* b, int m, double theta, double* y) {
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale += fabs(a[i]) + (i + 1 < m ? fabs(b[i]) : 0.0);
  const double shift = theta - 1e-13 * (scale > 0.0 ? scale : 1.0);
  for (int i = 0; i < m; ++i) y[i] = 1.0;
  for (int it = 0; it < 3; ++it) {
    tri_solve(a, b, m, shift, y);
    double n = 0.0;
    for (int i = 0; i < m; ++i) n += y[i] * y[i];
    n = sqrt(n);
    for (int i = 0; i < m; ++i) y[i] /= n;
  }
  /* sign: largest |component| positive */
  int best = 0;
  for (int i = 1; i < m; ++i)
    if (fabs(y[i]) > fabs(y[best])) best = i;
  if (y[best] < 0.0)
    for (int i = 0; i < m; ++i) y[i] = -y[i];
}

/* ---------------------------------------------------------------------------------- */
/* exported                                                                            */
/* ---------------------------------------------------------------------------------- */
static double dotp(const double* u, const double* v, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
  return s;
}

/* dimension of the sector (or a negative code) */
int64_t mscheme_dim(int N, const int8_t* species, const int8_t* two_m, int Np, int Nn,
                    int two_M) {
  Sector S;
  double eps[64] = {0};
  const int rc = sector_build(&S, N, species, two_m, eps, 0, NULL, NULL, Np, Nn, two_M);
  const int64_t d = rc == 0 ? S.dim : rc;
  sector_free(&S);
  return d;
}

/* determinant masks of the basis in vector order (masks: dim entries) */
int mscheme_basis(int N, const int8_t* species, const int8_t* two_m, int Np, int Nn, int two_M,
                  uint64_t* masks) {
  Sector S;
  double eps[64] = {0};
  const int rc = sector_build(&S, N, species, two_m, eps, 0, NULL, NULL, Np, Nn, two_M);
  if (rc == 0)
    for (int64_t r = 0; r < S.dim; ++r) masks[r] = sector_mask(&S, r);
  sector_free(&S);
  return rc;
}

/* y = H x in the sector basis */
int mscheme_apply(int N, const int8_t* species, const int8_t* two_m, const double* eps,
                  int64_t n_v, const int32_t* v_idx, const double* v_val, int Np, int Nn,
                  int two_M, const double* x, double* y, int n_threads) {
  Sector S;
  const int rc = sector_build(&S, N, species, two_m, eps, n_v, v_idx, v_val, Np, Nn, two_M);
  if (rc == 0) apply_h(&S, x, y, n_threads);
  sector_free(&S);
  return rc;
}

/* lowest eigenpair; vec (optional, dim entries) receives the normalised Ritz vector.
 * info[0] = Lanczos steps, info[1] = dimension; out[0] = energy, out[1] = explicit
 * residual |H x - E x|, out[2] = the Lanczos residual estimate.  Returns 0, or < 0 for
 * invalid input, or 1 when max_iter was reached before the tolerance. */
int mscheme_lanczos(int N, const int8_t* species, const int8_t* two_m, const double* eps,
                    int64_t n_v, const int32_t* v_idx, const double* v_val, int Np, int Nn,
                    int two_M, int max_iter, double tol, int n_threads, double* vec,
                    int64_t* info, double* out) {
  Sector S;
  int rc = sector_build(&S, N, species, two_m, eps, n_v, v_idx, v_val, Np, Nn, two_M);
  if (rc != 0) {
    sector_free(&S);
    return rc;
  }
  const int64_t n = S.dim;
  if (n <= 0) {
    sector_free(&S);
    return -3;
  }
  if (max_iter > n) max_iter = (int)n;
  if (max_iter < 1) max_iter = 1;
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(max_iter + 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* a = (double*)malloc(sizeof(double) * (size_t)(max_iter + 1));
  double* b = (double*)malloc(sizeof(double) * (size_t)(max_iter + 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)(max_iter + 1));
  if (!V || !w || !a || !b || !y) {
    free(V);
    free(w);
    free(a);
    free(b);
    free(y);
    sector_free(&S);
    return -4;
  }
  /* start vector: 1 + 0.5 sin(r + 1), normalised (overlaps every eigenvector in general) */
  double nr = 0.0;
  for (int64_t r = 0; r < n; ++r) {
    V[r] = 1.0 + 0.5 * sin((double)r + 1.0);
    nr += V[r] * V[r];
  }
  nr = sqrt(nr);
  for (int64_t r = 0; r < n; ++r) V[r] /= nr;
  int m = 0;
  double theta = 0.0, theta_prev = 0.0, est = 0.0;
  rc = 1;
  for (int j = 0; j < max_iter; ++j) {
    double* vj = V + (size_t)j * (size_t)n;
    apply_h(&S, vj, w, n_threads);
    if (j > 0) {
      const double* vp = V + (size_t)(j - 1) * (size_t)n;
      for (int64_t r = 0; r < n; ++r) w[r] -= b[j - 1] * vp[r];
    }
    a[j] = dotp(vj, w, n);
    for (int64_t r = 0; r < n; ++r) w[r] -= a[j] * vj[r];
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i <= j; ++i) {
        const double* vi = V + (size_t)i * (size_t)n;
        const double c = dotp(vi, w, n);
        for (int64_t r = 0; r < n; ++r) w[r] -= c * vi[r];
      }
    b[j] = sqrt(dotp(w, w, n));
    m = j + 1;
    theta = tri_lowest(a, b, m);
    tri_vector(a, b, m, theta, y);
    est = fabs(b[j] * y[m - 1]);
    const int settled = j > 0 && fabs(theta - theta_prev) < 1e-13 * (1.0 + fabs(theta));
    theta_prev = theta;
    if ((est <= tol && settled) || b[j] <= 1e-300 || m == n) {
      rc = 0;
      break;
    }
    double* vn = V + (size_t)(j + 1) * (size_t)n;
    for (int64_t r = 0; r < n; ++r) vn[r] = w[r] / b[j];
  }
  /* Ritz vector and its explicit residual */
  for (int64_t r = 0; r < n; ++r) w[r] = 0.0;
  for (int i = 0; i < m; ++i) {
    const double* vi = V + (size_t)i * (size_t)n;
    for (int64_t r = 0; r < n; ++r) w[r] += y[i] * vi[r];
  }
  double nx = sqrt(dotp(w, w, n));
  for (int64_t r = 0; r < n; ++r) w[r] /= nx;
  double* hx = V;   /* reuse the first Lanczos vector's storage */
  apply_h(&S, w, hx, n_threads);
  double res = 0.0;
  for (int64_t r = 0; r < n; ++r) {
    const double d = hx[r] - theta * w[r];
    res += d * d;
  }
  if (vec) memcpy(vec, w, sizeof(double) * (size_t)n);
  info[0] = m;
  info[1] = n;
  out[0] = theta;
  out[1] = sqrt(res);
  out[2] = est;
  free(V);
  free(w);
  free(a);
  free(b);
  free(y);
  sector_free(&S);
  return rc;
}
