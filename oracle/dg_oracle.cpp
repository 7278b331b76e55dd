// dg_oracle.cpp -- plain, slow, single-threaded FP64 reference of the BDD
// Lagrange-dual solver of DOGE-Train (Abbas & Swoboda, arXiv 2205.11638).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
// leg of bench.py may load this library.  It shares no code, header, table or
// helper with the CUDA path (paper_2205_11638_gb300/csrc) and must never be
// used as a fallback for it.
//
// What it follows, passage by passage:
//   * Def. 1 (binary program BP) and the remark after it: every linear row
//     a_j^T x {<=,=,>=} b_j is one subproblem X_j            (Sec. 3.1)
//   * Def. 2 (Lagrangean dual D, E^j, J_i)                    (Sec. 3.1, eq. 1)
//   * Alg. 1 "Generalized Min-Marginal Averaging" and its BlockUpdate
//                                                              (Sec. 3.2)
//   * Alg. 2 "BlockUpdate backpropagation", used literally with explicit
//     minimiser vectors s^j(i,beta)                            (Sec. 3.3)
//   * App. B: BDD representation, shortest-path costs SP(r,v), SP(v,T) and
//     the min-marginal formula via shortest paths              (App. B)
//   * the loss L(lambda) = sum_j E^j and its gradient, the minimising
//     assignment of each subproblem                            (Sec. 3.5, eq. 3)
//   * the non-parametric update of eq. 2                        (Sec. 3.4)
//   * the output transforms of the parameter predictor: softmax of the
//     averaging weights over J_i, sigmoid of the damping, centring of theta
//                                                               (Sec. 3.5, Alg. 3)
//   * the smoothed subproblems of the feature table and their gradients
//                                                    (App. C, hand-crafted features)
//
//   R12 the smoothed subproblem is printed as alpha log sum_x exp(<lambda,x>/alpha),
//       a soft-max; as the smoothing of a minimisation it is read as
//       E_a(lambda) = -a log sum_{x in X_j} exp(-<lambda, x>/a), which tends to
//       E^j as a -> 0; its gradient is the vector of marginals P(x_i = 1).
//
// Readings where the paper is silent or garbled (each one is also listed in
// the design notes of the repository):
//   R1  sum_{k in J_i} M^old_ik in the lambda update is a snapshot taken at the
//       start of each sweep (the feasibility proof of Prop. 1 only closes if
//       every (i,j) of a sweep sees the same sum).
//   R2  the invariant of the proof of Prop. 1 reads sum_j (lambda_ij + M_ij) = c_i.
//   R3  lower bound while M != 0: sum_j E^j(lambda) + sum_i min(0, S_i) with
//       S_i = sum_j M_ij, plus min(0, c_i) for variables in no subproblem.
//   R4  initial lambda_ij = c_i / |J_i|, M = 0.
//   R5  block k of a sweep = the k-th variable (hop) of every BDD; variables of
//       a BDD in ascending id order.
//   R6  omega in [0,1], alpha >= 0 (closed ranges).
//   R7  Alg. 2: the gradient of M^old_ij is sum_k alpha_ik * dlambda^new_ik for
//       every j; omega's gradient uses the stored (m1 - m0), not M/omega.
//   R8  a row that fixes one of its variables (some min-marginal infinite) is
//       rejected (status 5); an infeasible row is rejected (status 4).
//   R9  ties: relaxation of SP(r,.) keeps the in-arc with the smallest
//       (parent rank, beta); SP(.,T) keeps the 0-arc; the min-marginal argmin
//       over P_i keeps the smallest node rank; the loss argmin walks 0-arcs on
//       ties.
//   R10 canonical node order at each level: ascending (lo code, hi code) with
//       bottom = -2, top = -1, children as ranks on the next level.
//
// One "iteration" is a forward sweep over blocks B_1..B_u followed by a
// backward sweep B_u..B_1.  State vectors are indexed by CSR slot: row j,
// position h within the row (columns strictly ascending).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <set>
#include <string>
#include <utility>
#include <vector>

namespace {

const int BOT = -2;
const int TOP = -1;
const double INF = std::numeric_limits<double>::infinity();

// One subproblem as a quasi-reduced BDD (App. B): level h holds the nodes P_i
// of the h-th variable of the row; every r-T path meets exactly one node per
// level.  Children are ranks on level h+1, or BOT / TOP.
struct Bdd {
    int k = 0;
    std::vector<int> level_start;  // k+1 entries
    std::vector<int> lo, hi;       // per node
};

struct Problem {
    int n = 0;
    int64_t m = 0;
    int num_inst = 1;
    std::vector<int64_t> row_ptr;
    std::vector<int> col;
    std::vector<double> c;
    std::vector<int64_t> inst_row_ptr;
    std::vector<int> inst_var_ptr;
    std::vector<Bdd> bdd;
    std::vector<int> deg;  // |J_i|
    std::vector<int> slot_row;
};

std::string g_err;

bool satisfied(int64_t s, int sense, int64_t b) {
    if (sense == 0) return s <= b;
    if (sense == 1) return s >= b;
    return s == b;
}

// Builds the BDD of one row by dynamic programming over partial sums: a
// top-down pass collects the partial sums reachable at every level, a
// bottom-up pass gives every (level, partial sum) the code of its residual
// function.  Two partial sums with the same (lo code, hi code) pair have the
// same residual function and become one node.  Returns 0, 4 (infeasible) or
// 5 (forced variable).
int build_bdd(const int* a, int k, int sense, int64_t b, Bdd& B) {
    std::vector<std::vector<int64_t>> sums(k + 1);
    sums[0].push_back(0);
    for (int h = 0; h < k; ++h) {
        std::set<int64_t> next;
        for (int64_t s : sums[h]) {
            next.insert(s);
            next.insert(s + a[h]);
        }
        sums[h + 1].assign(next.begin(), next.end());
    }
    std::vector<std::map<int64_t, int>> code(k + 1);
    for (int64_t s : sums[k]) code[k][s] = satisfied(s, sense, b) ? TOP : BOT;

    std::vector<std::vector<std::pair<int, int>>> level_nodes(k);
    for (int h = k - 1; h >= 0; --h) {
        std::map<std::pair<int, int>, int> rank;
        std::vector<std::pair<int, int>> key_of(sums[h].size());
        for (size_t q = 0; q < sums[h].size(); ++q) {
            int64_t s = sums[h][q];
            std::pair<int, int> key(code[h + 1].at(s), code[h + 1].at(s + a[h]));
            key_of[q] = key;
            if (!(key.first == BOT && key.second == BOT)) rank[key] = 0;
        }
        int r = 0;
        for (auto& kv : rank) {
            kv.second = r++;
            level_nodes[h].push_back(kv.first);
        }
        for (size_t q = 0; q < sums[h].size(); ++q) {
            const auto& key = key_of[q];
            code[h][sums[h][q]] = (key.first == BOT && key.second == BOT) ? BOT : rank[key];
        }
    }
    if (code[0].at(0) == BOT) return 4;

    B.k = k;
    B.level_start.assign(k + 1, 0);
    B.lo.clear();
    B.hi.clear();
    for (int h = 0; h < k; ++h) {
        B.level_start[h] = (int)B.lo.size();
        bool any_lo = false, any_hi = false;
        for (const auto& key : level_nodes[h]) {
            B.lo.push_back(key.first);
            B.hi.push_back(key.second);
            any_lo |= key.first != BOT;
            any_hi |= key.second != BOT;
        }
        if (!any_lo || !any_hi) return 5;
    }
    B.level_start[k] = (int)B.lo.size();
    return 0;
}

// SP(v, T) for every node under lambda (App. B): bottom-up min-sum, bottom
// children skipped.
void cost_to_top(const Bdd& B, const double* lam, std::vector<double>& t) {
    t.assign(B.lo.size(), INF);
    for (int h = B.k - 1; h >= 0; --h) {
        for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v) {
            double best = INF;
            if (B.lo[v] != BOT) {
                double tl = B.lo[v] == TOP ? 0.0 : t[B.level_start[h + 1] + B.lo[v]];
                best = tl;
            }
            if (B.hi[v] != BOT) {
                double th = B.hi[v] == TOP ? 0.0 : t[B.level_start[h + 1] + B.hi[v]];
                best = std::min(best, lam[h] + th);
            }
            t[v] = best;
        }
    }
}

// SP(r, v) for every node under lambda: top-down min-sum.
void cost_from_root(const Bdd& B, const double* lam, std::vector<double>& d) {
    d.assign(B.lo.size(), INF);
    d[0] = 0.0;
    for (int h = 0; h + 1 < B.k; ++h) {
        for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v) {
            if (B.lo[v] >= 0) {
                int w = B.level_start[h + 1] + B.lo[v];
                d[w] = std::min(d[w], d[v]);
            }
            if (B.hi[v] >= 0) {
                int w = B.level_start[h + 1] + B.hi[v];
                d[w] = std::min(d[w], d[v] + lam[h]);
            }
        }
    }
}

double child_cost(const Bdd& B, int h, int child, const std::vector<double>& t) {
    return child == TOP ? 0.0 : t[B.level_start[h + 1] + child];
}

// Min-marginals of level h by the shortest-path formula of App. B:
//   m^beta = min over v in P_i with a beta-arc of SP(r,v) + beta*lambda + SP(s^beta(v),T).
// d must be valid on level h and t on level h+1.
void level_min_marginals(const Bdd& B, int h, double lam_h, const std::vector<double>& d,
                         const std::vector<double>& t, double& m0, double& m1) {
    double b0 = INF, b1 = INF;
    for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v) {
        if (B.lo[v] != BOT) b0 = std::min(b0, d[v] + child_cost(B, h, B.lo[v], t));
        if (B.hi[v] != BOT) b1 = std::min(b1, d[v] + child_cost(B, h, B.hi[v], t));
    }
    m0 = b0;
    m1 = lam_h + b1;
}

// Relaxes SP(r, .) of level h+1 from level h (Alg. 1 keeps SP(r, .) current
// while a forward sweep advances, App. B).
void relax_level(const Bdd& B, int h, double lam_h, std::vector<double>& d) {
    if (h + 1 >= B.k) return;
    for (int w = B.level_start[h + 1]; w < B.level_start[h + 2]; ++w) d[w] = INF;
    for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v) {
        if (B.lo[v] >= 0) {
            int w = B.level_start[h + 1] + B.lo[v];
            d[w] = std::min(d[w], d[v]);
        }
        if (B.hi[v] >= 0) {
            int w = B.level_start[h + 1] + B.hi[v];
            d[w] = std::min(d[w], d[v] + lam_h);
        }
    }
}

// Recomputes SP(v, T) of level h from level h+1 (kept current while a
// backward sweep descends).
void retop_level(const Bdd& B, int h, double lam_h, std::vector<double>& t) {
    for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v) {
        double best = INF;
        if (B.lo[v] != BOT) best = child_cost(B, h, B.lo[v], t);
        if (B.hi[v] != BOT) best = std::min(best, lam_h + child_cost(B, h, B.hi[v], t));
        t[v] = best;
    }
}

std::vector<double> snapshot_S(const Problem& P, const double* M) {
    std::vector<double> S(P.n, 0.0);
    for (size_t s = 0; s < P.col.size(); ++s) S[P.col[s]] += M[s];
    return S;
}

// One sweep of Alg. 1: the forward sweep runs blocks B_1..B_u, the backward
// sweep B_u..B_1.  Each block performs BlockUpdate for every subproblem that
// has a variable in it:
//   M^new_ij      = omega_ij (m1_ij - m0_ij)
//   lambda^new_ij = lambda^old_ij - M^new_ij + alpha_ij * S^in_i
// with S^in the snapshot of reading R1.  d and t are the SP(r,.) and SP(.,T)
// arrays of every BDD; the sweep keeps the one of its direction current.
void sweep(const Problem& P, bool forward, double* lam, double* M, const double* omega,
           const double* alpha, std::vector<std::vector<double>>& d,
           std::vector<std::vector<double>>& t) {
    std::vector<double> S = snapshot_S(P, M);
    // BDDs are independent within a sweep (reading R1); the pragma only acts
    // in the separately built all-cores timing copy of this file
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t j = 0; j < P.m; ++j) {
        const Bdd& B = P.bdd[j];
        const int64_t base = P.row_ptr[j];
        double* lj = lam + base;
        if (forward) {
            d[j].assign(B.lo.size(), INF);
            d[j][0] = 0.0;
        }
        for (int q = 0; q < B.k; ++q) {
            int h = forward ? q : B.k - 1 - q;
            int64_t s = base + h;
            double m0, m1;
            level_min_marginals(B, h, lj[h], d[j], t[j], m0, m1);
            double Mn = omega[s] * (m1 - m0);
            lj[h] = lj[h] - Mn + alpha[s] * S[P.col[s]];
            M[s] = Mn;
            if (forward)
                relax_level(B, h, lj[h], d[j]);
            else
                retop_level(B, h, lj[h], t[j]);
        }
    }
}

void full_iterate(const Problem& P, double* lam, double* M, const double* omega, const double* alpha,
                  int iters, double* lb_trace);

double lower_bound_impl(const Problem& P, const double* lam, const double* M, double* per_inst) {
    std::vector<double> S = snapshot_S(P, M);
    std::vector<double> inst(P.num_inst, 0.0);
    std::vector<double> t;
    for (int k = 0; k < P.num_inst; ++k) {
        double acc = 0.0;
        for (int64_t j = P.inst_row_ptr[k]; j < P.inst_row_ptr[k + 1]; ++j) {
            cost_to_top(P.bdd[j], lam + P.row_ptr[j], t);
            acc += t[0];  // E^j = SP(r, T)
        }
        for (int i = P.inst_var_ptr[k]; i < P.inst_var_ptr[k + 1]; ++i)
            acc += P.deg[i] > 0 ? std::min(0.0, S[i]) : std::min(0.0, P.c[i]);
        inst[k] = acc;
    }
    double tot = 0.0;
    for (int k = 0; k < P.num_inst; ++k) {
        if (per_inst) per_inst[k] = inst[k];
        tot += inst[k];
    }
    return tot;
}

void full_iterate(const Problem& P, double* lam, double* M, const double* omega, const double* alpha,
                  int iters, double* lb_trace) {
    std::vector<std::vector<double>> d(P.m), t(P.m);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t j = 0; j < P.m; ++j) cost_to_top(P.bdd[j], lam + P.row_ptr[j], t[j]);
    for (int it = 0; it < iters; ++it) {
        sweep(P, true, lam, M, omega, alpha, d, t);
        sweep(P, false, lam, M, omega, alpha, d, t);
        if (lb_trace) lb_trace[it] = lower_bound_impl(P, lam, M, nullptr);
    }
}

// Minimising assignment of one subproblem with x_h = beta (Alg. 2 line
// "compute minimizers"), under lambda of that subproblem.  The path is the
// one the routed shortest-path gradients follow (reading R9): the argmin node
// v* on level h (smallest rank), the argmin in-arcs from v* back to the root
// (smallest (parent rank, beta)) and the argmin out-arcs from s^beta(v*) to
// the top (0-arc on ties).
void minimiser(const Bdd& B, const double* lam, int h, int beta, std::vector<int>& x) {
    std::vector<double> d, t;
    cost_from_root(B, lam, d);
    cost_to_top(B, lam, t);
    x.assign(B.k, 0);
    int vstar = -1;
    double best = INF;
    for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v) {
        int ch = beta ? B.hi[v] : B.lo[v];
        if (ch == BOT) continue;
        double val = d[v] + child_cost(B, h, ch, t);
        if (val < best) {
            best = val;
            vstar = v;
        }
    }
    x[h] = beta;
    // prefix: walk argmin in-arcs back to the root
    int w = vstar;
    for (int g = h; g >= 1; --g) {
        int wr = w - B.level_start[g];
        int bp = -1, bb = -1;
        double bv = INF;
        for (int p = B.level_start[g - 1]; p < B.level_start[g]; ++p) {
            for (int bt = 0; bt < 2; ++bt) {
                int ch = bt ? B.hi[p] : B.lo[p];
                if (ch != wr) continue;
                double val = d[p] + (bt ? lam[g - 1] : 0.0);
                if (val < bv) {
                    bv = val;
                    bp = p;
                    bb = bt;
                }
            }
        }
        x[g - 1] = bb;
        w = bp;
    }
    // suffix: walk argmin out-arcs to the top
    int ch = beta ? B.hi[vstar] : B.lo[vstar];
    for (int g = h + 1; g < B.k; ++g) {
        int v = B.level_start[g] + ch;
        bool take0 = false;
        if (B.lo[v] != BOT) {
            take0 = B.hi[v] == BOT ||
                    child_cost(B, g, B.lo[v], t) <= lam[g] + child_cost(B, g, B.hi[v], t);
        }
        x[g] = take0 ? 0 : 1;
        ch = take0 ? B.lo[v] : B.hi[v];
    }
}

}  // namespace

extern "C" {

const char* orc_last_error(void) { return g_err.c_str(); }

// Creates a problem from CSR rows.  sense: 0 '<=', 1 '>=', 2 '='.  Columns of
// every row must be strictly ascending.  Status: 0 ok, 1 invalid input,
// 4 infeasible row, 5 row forcing a variable.
int orc_create(int n, int64_t m, const int64_t* row_ptr, const int32_t* col, const int32_t* coef,
               const int8_t* sense, const int32_t* rhs, const double* c, int num_inst,
               const int64_t* inst_row_ptr, const int32_t* inst_var_ptr, void** out) {
    *out = nullptr;
    Problem* P = new Problem();
    P->n = n;
    P->m = m;
    P->num_inst = num_inst;
    P->row_ptr.assign(row_ptr, row_ptr + m + 1);
    P->col.assign(col, col + row_ptr[m]);
    P->c.assign(c, c + n);
    if (num_inst <= 1 || !inst_row_ptr || !inst_var_ptr) {
        P->num_inst = 1;
        P->inst_row_ptr = {0, m};
        P->inst_var_ptr = {0, n};
    } else {
        P->inst_row_ptr.assign(inst_row_ptr, inst_row_ptr + num_inst + 1);
        P->inst_var_ptr.assign(inst_var_ptr, inst_var_ptr + num_inst + 1);
    }
    P->deg.assign(n, 0);
    P->bdd.resize(m);
    P->slot_row.resize(row_ptr[m]);
    for (int64_t j = 0; j < m; ++j) {
        int64_t b0 = row_ptr[j], b1 = row_ptr[j + 1];
        if (b1 <= b0) {
            g_err = "empty row " + std::to_string(j);
            delete P;
            return 1;
        }
        for (int64_t s = b0; s < b1; ++s) {
            if (col[s] < 0 || col[s] >= n || (s > b0 && col[s] <= col[s - 1])) {
                g_err = "row " + std::to_string(j) + ": columns must be ascending ids in [0,n)";
                delete P;
                return 1;
            }
            P->deg[col[s]]++;
            P->slot_row[s] = (int)j;
        }
        std::vector<int> a(coef + b0, coef + b1);
        int st = build_bdd(a.data(), (int)(b1 - b0), sense[j], rhs[j], P->bdd[j]);
        if (st != 0) {
            g_err = std::string(st == 4 ? "infeasible" : "variable-forcing") + " row " + std::to_string(j);
            delete P;
            return st;
        }
    }
    *out = P;
    return 0;
}

void orc_destroy(void* p) { delete static_cast<Problem*>(p); }

int64_t orc_num_slots(void* p) { return (int64_t) static_cast<Problem*>(p)->col.size(); }

int64_t orc_num_nodes(void* p) {
    int64_t s = 0;
    for (auto& B : static_cast<Problem*>(p)->bdd) s += (int64_t)B.lo.size();
    return s;
}

// Structure of BDD j: level_start (k+1 ints) and lo/hi codes per node.
int orc_bdd_size(void* p, int64_t j) { return (int)static_cast<Problem*>(p)->bdd[j].lo.size(); }

void orc_bdd_export(void* p, int64_t j, int32_t* level_start, int32_t* lo, int32_t* hi) {
    const Bdd& B = static_cast<Problem*>(p)->bdd[j];
    for (int h = 0; h <= B.k; ++h) level_start[h] = B.level_start[h];
    for (size_t v = 0; v < B.lo.size(); ++v) {
        lo[v] = B.lo[v];
        hi[v] = B.hi[v];
    }
}

// Initial dual variables (reading R4): lambda_ij = c_i / |J_i|, M = 0.
void orc_init_lambda(void* p, double* lam, double* M) {
    Problem* P = static_cast<Problem*>(p);
    for (size_t s = 0; s < P->col.size(); ++s) {
        lam[s] = P->c[P->col[s]] / P->deg[P->col[s]];
        M[s] = 0.0;
    }
}

// Runs `iters` iterations of Alg. 1 in place.  lb_trace (nullable) receives
// the bound of reading R3 after every iteration.
void orc_iterate(void* p, double* lam, double* M, const double* omega, const double* alpha, int iters,
                 double* lb_trace) {
    full_iterate(*static_cast<Problem*>(p), lam, M, omega, alpha, iters, lb_trace);
}

// Runs one sweep (forward = 1 or backward = 0) from scratch: SP(.,T) is
// recomputed from lambda first (a backward sweep also needs SP(r,.), which is
// recomputed from lambda too).  Used by the per-sweep invariant pins.
void orc_sweep(void* p, int forward, double* lam, double* M, const double* omega, const double* alpha) {
    Problem& P = *static_cast<Problem*>(p);
    std::vector<std::vector<double>> d(P.m), t(P.m);
    for (int64_t j = 0; j < P.m; ++j) {
        cost_to_top(P.bdd[j], lam + P.row_ptr[j], t[j]);
        cost_from_root(P.bdd[j], lam + P.row_ptr[j], d[j]);
    }
    sweep(P, forward != 0, lam, M, omega, alpha, d, t);
}

// Min-marginals m0, m1 of every slot under lambda, by the shortest-path
// formula of App. B (no update).
void orc_min_marginals(void* p, const double* lam, double* m0, double* m1) {
    Problem& P = *static_cast<Problem*>(p);
    std::vector<double> d, t;
    for (int64_t j = 0; j < P.m; ++j) {
        const Bdd& B = P.bdd[j];
        const double* lj = lam + P.row_ptr[j];
        cost_from_root(B, lj, d);
        cost_to_top(B, lj, t);
        for (int h = 0; h < B.k; ++h)
            level_min_marginals(B, h, lj[h], d, t, m0[P.row_ptr[j] + h], m1[P.row_ptr[j] + h]);
    }
}

// Lower bound of reading R3; per_inst (nullable) receives one value per
// instance.  E_out (nullable) receives E^j(lambda) per row.
double orc_lower_bound(void* p, const double* lam, const double* M, double* per_inst, double* E_out) {
    Problem& P = *static_cast<Problem*>(p);
    if (E_out) {
        std::vector<double> t;
        for (int64_t j = 0; j < P.m; ++j) {
            cost_to_top(P.bdd[j], lam + P.row_ptr[j], t);
            E_out[j] = t[0];
        }
    }
    return lower_bound_impl(P, lam, M, per_inst);
}

// Gradient of the bound of reading R3 (eq. 3 plus the unary term): the
// minimising assignment of every subproblem (0-arc on ties) for lambda, and
// [S_i < 0] for every M_ij.
void orc_lb_seed(void* p, const double* lam, const double* M, double* g_lam, double* g_M) {
    Problem& P = *static_cast<Problem*>(p);
    std::vector<double> S = snapshot_S(P, M);
    std::vector<double> t;
    for (int64_t j = 0; j < P.m; ++j) {
        const Bdd& B = P.bdd[j];
        const double* lj = lam + P.row_ptr[j];
        cost_to_top(B, lj, t);
        int ch = 0;
        for (int h = 0; h < B.k; ++h) {
            int v = B.level_start[h] + ch;
            bool take0 = false;
            if (B.lo[v] != BOT)
                take0 = B.hi[v] == BOT || child_cost(B, h, B.lo[v], t) <= lj[h] + child_cost(B, h, B.hi[v], t);
            g_lam[P.row_ptr[j] + h] = take0 ? 0.0 : 1.0;
            ch = take0 ? B.lo[v] : B.hi[v];
        }
    }
    for (size_t s = 0; s < P.col.size(); ++s) g_M[s] = S[P.col[s]] < 0.0 ? 1.0 : 0.0;
}

// Minimising assignment of row j with its h-th variable fixed to beta, under
// the slot values lam_row (|I_j| entries); tie rules of reading R9.
void orc_minimiser(void* p, int64_t j, const double* lam_row, int h, int beta, int32_t* x) {
    std::vector<int> xv;
    minimiser(static_cast<Problem*>(p)->bdd[j], lam_row, h, beta, xv);
    for (size_t q = 0; q < xv.size(); ++q) x[q] = xv[q];
}

// Backpropagation through `iters` iterations of Alg. 1 (Alg. 2 applied block
// by block, newest first).  Inputs: the state (lam0, M0) the iterations start
// from, omega and alpha per slot, the gradients g_lamT, g_MT of the loss with
// respect to the final state.  Outputs: gradients with respect to lam0, M0,
// omega and alpha (accumulated over all blocks, as Alg. 2 does for parameters
// shared by several iterations).
void orc_backward(void* p, const double* lam0, const double* M0, const double* omega, const double* alpha,
                  int iters, const double* g_lamT, const double* g_MT, double* g_lam0, double* g_M0,
                  double* g_omega, double* g_alpha) {
    Problem& P = *static_cast<Problem*>(p);
    const size_t N = P.col.size();
    const int nsweeps = 2 * iters;
    // forward replay, keeping lambda and S^in at the start of every sweep
    std::vector<std::vector<double>> lam_at(nsweeps + 1), S_at(nsweeps);
    std::vector<double> lam(lam0, lam0 + N), M(M0, M0 + N);
    {
        std::vector<std::vector<double>> d(P.m), t(P.m);
        for (int64_t j = 0; j < P.m; ++j) cost_to_top(P.bdd[j], lam.data() + P.row_ptr[j], t[j]);
        for (int s = 0; s < nsweeps; ++s) {
            lam_at[s] = lam;
            S_at[s] = snapshot_S(P, M.data());
            sweep(P, s % 2 == 0, lam.data(), M.data(), omega, alpha, d, t);
        }
        lam_at[nsweeps] = lam;
    }
    std::vector<double> gl(g_lamT, g_lamT + N), gM(g_MT, g_MT + N);
    std::fill(g_omega, g_omega + N, 0.0);
    std::fill(g_alpha, g_alpha + N, 0.0);
    std::vector<double> cur, dd, tt;
    std::vector<int> s1, s0;
    for (int s = nsweeps - 1; s >= 0; --s) {
        const bool forward = s % 2 == 0;
        std::vector<double> Sdot(P.n, 0.0);
        for (int64_t j = 0; j < P.m; ++j) {
            const Bdd& B = P.bdd[j];
            const int64_t base = P.row_ptr[j];
            const double* lo_ = lam_at[s].data() + base;
            const double* ln_ = lam_at[s + 1].data() + base;
            // blocks of this sweep in reverse order
            for (int q = B.k - 1; q >= 0; --q) {
                int h = forward ? q : B.k - 1 - q;
                // lambda_{.j} as block h saw it: slots updated earlier in the
                // sweep hold their new value
                cur.assign(B.k, 0.0);
                for (int g = 0; g < B.k; ++g) {
                    bool updated_before = forward ? (g < h) : (g > h);
                    cur[g] = updated_before ? ln_[g] : lo_[g];
                }
                const int64_t sl = base + h;
                const int i = P.col[sl];
                const double glam = gl[sl];
                Sdot[i] += alpha[sl] * glam;
                g_alpha[sl] += glam * S_at[s][i];
                const double Mdot = gM[sl] - glam;
                cost_from_root(B, cur.data(), dd);
                cost_to_top(B, cur.data(), tt);
                double m0, m1;
                level_min_marginals(B, h, cur[h], dd, tt, m0, m1);
                g_omega[sl] += Mdot * (m1 - m0);
                minimiser(B, cur.data(), h, 1, s1);
                minimiser(B, cur.data(), h, 0, s0);
                for (int g = 0; g < B.k; ++g) gl[base + g] += Mdot * omega[sl] * (double)(s1[g] - s0[g]);
            }
        }
        for (size_t sl = 0; sl < N; ++sl) gM[sl] = Sdot[P.col[sl]];
    }
    std::copy(gl.begin(), gl.end(), g_lam0);
    std::copy(gM.begin(), gM.end(), g_M0);
}

// Non-parametric update (eq. 2): lambda_ij += theta_ij - mean_{k in J_i} theta_ik.
void orc_nonparam_update(void* p, double* lam, const double* theta) {
  Problem& P = *static_cast<Problem*>(p);
  std::vector<double> sum(P.n, 0.0);
  for (size_t s = 0; s < P.col.size(); ++s) sum[P.col[s]] += theta[s];
  for (size_t s = 0; s < P.col.size(); ++s) lam[s] += theta[s] - sum[P.col[s]] / P.deg[P.col[s]];
}

// Output transforms of Alg. 3: alpha_i. = softmax(alpha_hat_i.) over J_i,
// omega = sigmoid(omega_hat), theta_i. = theta_hat_i. - mean over J_i.
void orc_param_transform(void* p, const double* alpha_hat, const double* omega_hat, const double* theta_hat,
                         double* alpha, double* omega, double* theta) {
  Problem& P = *static_cast<Problem*>(p);
  const size_t N = P.col.size();
  std::vector<double> mx(P.n, -INF), z(P.n, 0.0), tsum(P.n, 0.0);
  for (size_t s = 0; s < N; ++s) mx[P.col[s]] = std::max(mx[P.col[s]], alpha_hat[s]);
  for (size_t s = 0; s < N; ++s) {
    z[P.col[s]] += std::exp(alpha_hat[s] - mx[P.col[s]]);
    tsum[P.col[s]] += theta_hat[s];
  }
  for (size_t s = 0; s < N; ++s) {
    const int i = P.col[s];
    alpha[s] = std::exp(alpha_hat[s] - mx[i]) / z[i];
    omega[s] = 1.0 / (1.0 + std::exp(-omega_hat[s]));
    theta[s] = theta_hat[s] - tsum[i] / P.deg[i];
  }
}

// Backpropagation through orc_param_transform: the Jacobian of the softmax
// of a variable's weights, the derivative of the sigmoid, and the centring
// (its own adjoint).
void orc_param_transform_backward(void* p, const double* alpha, const double* omega, const double* g_alpha,
                                  const double* g_omega, const double* g_theta, double* g_alpha_hat,
                                  double* g_omega_hat, double* g_theta_hat) {
  Problem& P = *static_cast<Problem*>(p);
  const size_t N = P.col.size();
  std::vector<double> dot(P.n, 0.0), gsum(P.n, 0.0);
  for (size_t s = 0; s < N; ++s) {
    dot[P.col[s]] += alpha[s] * g_alpha[s];
    gsum[P.col[s]] += g_theta[s];
  }
  for (size_t s = 0; s < N; ++s) {
    const int i = P.col[s];
    g_alpha_hat[s] = alpha[s] * (g_alpha[s] - dot[i]);
    g_omega_hat[s] = g_omega[s] * omega[s] * (1.0 - omega[s]);
    g_theta_hat[s] = g_theta[s] - gsum[i] / P.deg[i];
  }
}

// Smoothed subproblems (reading R12) by log-sum-exp over the BDD's paths:
// B(v) = log sum over v-T paths of exp(-cost/a), F(v) the same over r-v
// paths; log Z = B(root); E_a = -a log Z; the marginal of slot h is
// sum over level-h nodes with a 1-arc of exp(F(v) - lambda_h/a + B(s1(v)) - log Z).
static double lse(double x, double y) {
  if (x == -INF) return y;
  if (y == -INF) return x;
  const double m = std::max(x, y);
  return m + std::log(std::exp(x - m) + std::exp(y - m));
}

void orc_smoothed(void* p, const double* lam, double a, double* E_a, double* marg) {
  Problem& P = *static_cast<Problem*>(p);
  for (int64_t j = 0; j < P.m; ++j) {
    const Bdd& B = P.bdd[j];
    const double* lj = lam + P.row_ptr[j];
    std::vector<double> bw(B.lo.size(), -INF), fw(B.lo.size(), -INF);
    auto child_b = [&](int h, int ch) { return ch == TOP ? 0.0 : (ch == BOT ? -INF : bw[B.level_start[h + 1] + ch]); };
    for (int h = B.k - 1; h >= 0; --h)
      for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v)
        bw[v] = lse(child_b(h, B.lo[v]), B.hi[v] == BOT ? -INF : -lj[h] / a + child_b(h, B.hi[v]));
    const double logZ = bw[0];
    if (E_a) E_a[j] = -a * logZ;
    fw[0] = 0.0;
    for (int h = 0; h < B.k; ++h) {
      double acc = -INF;
      for (int v = B.level_start[h]; v < B.level_start[h + 1]; ++v) {
        if (B.hi[v] != BOT) acc = lse(acc, fw[v] - lj[h] / a + child_b(h, B.hi[v]));
        if (h + 1 < B.k) {
          if (B.lo[v] >= 0) {
            int w = B.level_start[h + 1] + B.lo[v];
            fw[w] = lse(fw[w], fw[v]);
          }
          if (B.hi[v] >= 0) {
            int w = B.level_start[h + 1] + B.hi[v];
            fw[w] = lse(fw[w], fw[v] - lj[h] / a);
          }
        }
      }
      if (marg) marg[P.row_ptr[j] + h] = std::exp(acc - logZ);
    }
  }
}

}  // extern "C"
