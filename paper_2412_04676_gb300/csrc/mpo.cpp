// mpo.cpp -- Eq. 1 of arXiv:2412.04676 split at every cut of the chain.
//
// For the two-site step of Sec. II.B every cut k needs operator sets with
// H = sum_w O^L_w (x) O^R_w.  They are built here from the terms of Eq. 1:
//
//   H = sum_{ij,s} h_ij a+_is a_js + sum_{p<q, r<s} W_pqrs a+_p a+_q a_r a_s
//
// (p, q, r, s spin orbitals 2*orbital + spin; W_pqrs = V_pqrs - V_pqsr with
// V_pqrs = (p s|q r) delta(spin p, spin s) delta(spin q, spin r), chemist
// integrals).  Each term is put in orbital order (sign = permutation parity);
// in Jordan-Wigner form its factor on orbital y is (its operators on y, in
// order) times P^(operators right of y), P = (-1)^n.  The state of a term at
// cut k is I before its first operator, F after its last, P(placed ops) for
// one placed operator or two placed while k < ksw (normal operators of the
// left block), and S(remaining ops) otherwise (complementary sums: the
// coefficient is folded in on entering S or F).  ksw moves two-operator
// sets to the side holding fewer orbitals (up to a two-cut offset from the
// centre), which keeps the number of states O(min(k, L-k)^2) per cut.
#include "mpo.h"

#include <array>
#include <cmath>
#include <unordered_map>

namespace gbd {
namespace {

using Key = uint64_t;
constexpr Key KIND_I = 0, KIND_P = 1, KIND_S = 2, KIND_F = 3;

inline Key make_key(Key kind, int n, const int* ops) {
    Key k = (kind << 62) | (Key(n) << 60);
    for (int i = 0; i < n; ++i) k |= Key(ops[i] + 1) << (40 - 20 * i);
    return k;
}
inline Key kind_of(Key k) { return k >> 62; }
inline int nops_of(Key k) { return int((k >> 60) & 3); }
inline int op_of(Key k, int i) { return int((k >> (40 - 20 * i)) & 0xFFFFF) - 1; }

inline int op_code(int orb, int spin, int dag) { return (orb << 2) | (spin << 1) | dag; }

// (n, tsz) change of a creation (dag=1) or annihilation operator
inline Q op_charge(int code) {
    int spin = (code >> 1) & 1, dag = code & 1;
    int sz = spin == 0 ? 1 : -1;
    return dag ? Q{1, sz} : Q{-1, -sz};
}

using Mat = std::array<double, 16>;

Mat local_op(int code) {
    Mat c{};  // creation operator of the given spin, basis 0, up, dn, updn
    int spin = (code >> 1) & 1, dag = code & 1;
    if (spin == 0) {
        c[1 * 4 + 0] = 1.0;   // |0>  -> |up>
        c[3 * 4 + 2] = 1.0;   // |dn> -> |updn>
    } else {
        c[2 * 4 + 0] = 1.0;   // |0>  -> |dn>
        c[3 * 4 + 1] = -1.0;  // |up> -> -|updn>
    }
    if (dag) return c;
    Mat t{};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) t[i * 4 + j] = c[j * 4 + i];
    return t;
}

Mat matmul(const Mat& a, const Mat& b) {
    Mat r{};
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k)
            if (a[i * 4 + k] != 0.0)
                for (int j = 0; j < 4; ++j) r[i * 4 + j] += a[i * 4 + k] * b[k * 4 + j];
    return r;
}

Mat identity() {
    Mat r{};
    for (int i = 0; i < 4; ++i) r[i * 5] = 1.0;
    return r;
}

Mat parity() {
    Mat r{};
    r[0] = 1.0; r[5] = -1.0; r[10] = -1.0; r[15] = 1.0;
    return r;
}

struct PairHash {
    size_t operator()(const std::pair<Key, Key>& p) const {
        uint64_t x = p.first * 0x9E3779B97F4A7C15ULL ^ (p.second + 0x632BE59BD9B4E019ULL + (p.first << 6));
        x ^= x >> 29;
        return size_t(x * 0xBF58476D1CE4E5B9ULL);
    }
};

struct EdgeAcc {
    Mat M{};
    bool coef = false;
};

struct Builder {
    int L, ksw;
    std::vector<std::unordered_map<std::pair<Key, Key>, EdgeAcc, PairHash>> edges;
    std::unordered_map<Key, std::pair<int, int>> alive;  // key -> [lo, hi] cuts
    Mat P = parity();

    void mark(Key k, int lo, int hi) {
        auto it = alive.find(k);
        if (it == alive.end()) {
            alive.emplace(k, std::make_pair(lo, hi));
        } else {
            it->second.first = std::min(it->second.first, lo);
            it->second.second = std::max(it->second.second, hi);
        }
    }

    void edge(int site, Key a, Key c, const Mat& M, double coef, bool with_coef) {
        auto& e = edges[site][{a, c}];
        if (with_coef) {
            for (int i = 0; i < 16; ++i) e.M[i] += coef * M[i];
            e.coef = true;
        } else {
            e.M = M;  // structural edges are identical for every term using them
        }
    }

    Key label(int placed, int m, int cut, const int* ops) const {
        if (placed == 0) return make_key(KIND_I, 0, ops);
        if (placed == m) return make_key(KIND_F, 0, ops);
        if (placed == 1) return make_key(KIND_P, 1, ops);
        if (placed == 2 && cut < ksw) return make_key(KIND_P, 2, ops);
        return make_key(KIND_S, m - placed, ops + placed);
    }

    // One term coef * o_0 o_1 ... o_{m-1} (as written).
    void term(double coef, const int* ops_in, int m) {
        int ops[4];
        for (int i = 0; i < m; ++i) ops[i] = ops_in[i];
        // stable insertion sort by orbital; each swap of operators on
        // different orbitals flips the sign
        double sign = 1.0;
        for (int i = 1; i < m; ++i) {
            int j = i;
            while (j > 0 && (ops[j - 1] >> 2) > (ops[j] >> 2)) {
                std::swap(ops[j - 1], ops[j]);
                sign = -sign;
                --j;
            }
        }
        const double c0 = coef * sign;
        Key prev = make_key(KIND_I, 0, ops);
        int prev_cut = 0;
        int placed = 0;
        int g = 0;
        while (g < m) {
            int y = ops[g] >> 2;
            int g1 = g;
            while (g1 < m && (ops[g1] >> 2) == y) ++g1;
            // the label of a two-placed term changes at cut ksw
            if (placed == 2 && m == 4 && prev_cut <= ksw - 1 && ksw - 1 < y) {
                Key nk = make_key(KIND_S, 2, ops + 2);
                mark(prev, prev_cut, ksw - 1);
                edge(ksw - 1, prev, nk, identity(), c0, true);
                prev = nk;
                prev_cut = ksw;
            }
            mark(prev, prev_cut, y);
            Mat M = identity();
            for (int i = g; i < g1; ++i) M = matmul(M, local_op(ops[i]));
            placed += g1 - g;
            int rem = m - placed;
            if (rem & 1) M = matmul(M, P);
            Key nk = label(placed, m, y + 1, ops);
            Key pk = kind_of(prev), nkk = kind_of(nk);
            bool with_coef = (nkk == KIND_S || nkk == KIND_F) && (pk == KIND_I || pk == KIND_P);
            edge(y, prev, nk, M, c0, with_coef);
            prev = nk;
            prev_cut = y + 1;
            g = g1;
        }
        mark(prev, prev_cut, L);
    }
};

int rem_parity(Key k) {
    Key kd = kind_of(k);
    if (kd == KIND_I || kd == KIND_F) return 0;
    return nops_of(k) & 1;  // P: placed count = remaining parity; S: remaining count
}

Q key_dq(Key k) {
    Key kd = kind_of(k);
    Q d{0, 0};
    if (kd == KIND_I || kd == KIND_F) return d;
    for (int i = 0; i < nops_of(k); ++i) d = d + op_charge(op_of(k, i));
    if (kd == KIND_S) d = Q{-d.n, -d.t};
    return d;
}

}  // namespace

void Mpo::build(int L_, const double* h, const double* eri, int ksw_) {
    L = L_;
    // The switch transform (normal pairs -> complementary pairs, an
    // O(k^2 (L-k)^2) coefficient contraction at one site) runs once per
    // half-sweep.  Default: one cut left of the centre, so the centre cut keeps
    // the minimal operator count and the two central positions do not enlarge
    // the switch site.
    ksw = ksw_ > 0 ? ksw_ : std::max(2, L / 2 - 1);
    Builder B;
    B.L = L;
    B.ksw = ksw;
    B.edges.resize(L);
    auto ERI = [&](int i, int j, int k, int l) { return eri[((size_t(i) * L + j) * L + k) * L + l]; };
    // one-body part
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            double v = h[size_t(i) * L + j];
            if (v == 0.0) continue;
            for (int s = 0; s < 2; ++s) {
                int ops[2] = {op_code(i, s, 1), op_code(j, s, 0)};
                B.term(v, ops, 2);
            }
        }
    // two-body part, antisymmetrised over p<q, r<s
    const int S = 2 * L;
    auto V = [&](int p, int q, int r, int s) -> double {
        if ((p & 1) != (s & 1) || (q & 1) != (r & 1)) return 0.0;
        return ERI(p >> 1, s >> 1, q >> 1, r >> 1);
    };
    for (int p = 0; p < S; ++p)
        for (int q = p + 1; q < S; ++q)
            for (int r = 0; r < S; ++r)
                for (int s = r + 1; s < S; ++s) {
                    // spin conservation: {spin p, spin q} == {spin r, spin s}
                    if (((p & 1) + (q & 1)) != ((r & 1) + (s & 1))) continue;
                    double w = V(p, q, r, s) - V(p, q, s, r);
                    if (w == 0.0) continue;
                    int ops[4] = {op_code(p >> 1, p & 1, 1), op_code(q >> 1, q & 1, 1),
                                  op_code(r >> 1, r & 1, 0), op_code(s >> 1, s & 1, 0)};
                    B.term(w, ops, 4);
                }
    // states alive at each cut, ascending key
    std::vector<std::vector<Key>> states(L + 1);
    for (auto& kv : B.alive)
        for (int c = kv.second.first; c <= kv.second.second; ++c) states[c].push_back(kv.first);
    std::vector<std::unordered_map<Key, int>> index(L + 1);
    dq.assign(L + 1, {});
    idxI.assign(L + 1, -1);
    idxF.assign(L + 1, -1);
    for (int c = 0; c <= L; ++c) {
        std::sort(states[c].begin(), states[c].end());
        index[c].reserve(states[c].size() * 2);
        for (size_t i = 0; i < states[c].size(); ++i) {
            Key k = states[c][i];
            index[c][k] = int(i);
            dq[c].push_back(key_dq(k));
            if (kind_of(k) == KIND_I) idxI[c] = int(i);
            if (kind_of(k) == KIND_F) idxF[c] = int(i);
        }
    }
    // pass-through: a state alive at cuts k and k+1 crosses orbital k
    Mat I4 = identity(), P4 = parity();
    for (auto& kv : B.alive) {
        for (int k = kv.second.first; k < kv.second.second; ++k) {
            auto key = std::make_pair(kv.first, kv.first);
            if (B.edges[k].find(key) == B.edges[k].end()) {
                EdgeAcc e;
                e.M = rem_parity(kv.first) ? P4 : I4;
                B.edges[k].emplace(key, e);
            }
        }
    }
    W.assign(L, {});
    for (int k = 0; k < L; ++k) {
        auto& out = W[k];
        for (auto& kv : B.edges[k]) {
            int a = index[k].at(kv.first.first);
            int c = index[k + 1].at(kv.first.second);
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    double v = kv.second.M[s * 4 + t];
                    if (v != 0.0) out.push_back({a, c, s, t, v});
                }
        }
        std::sort(out.begin(), out.end(), [](const MpoEntry& x, const MpoEntry& y) {
            if (x.c != y.c) return x.c < y.c;
            if (x.a != y.a) return x.a < y.a;
            if (x.s != y.s) return x.s < y.s;
            return x.t < y.t;
        });
    }
}

std::vector<double> Mpo::dense() const {
    GBD_REQUIRE(L >= 1 && L <= 5, GBD_ERR_ARG, "dense MPO contraction needs 1 <= L <= 5");
    int m = L / 2;
    // left[w] : 4^k x 4^k, right[w] : 4^(L-k) x 4^(L-k)
    std::vector<std::vector<double>> left(bond_dim(0));
    left[idxI[0]] = {1.0};
    int dl = 1;
    for (int k = 0; k < m; ++k) {
        std::vector<std::vector<double>> nl(bond_dim(k + 1));
        int nd = dl * 4;
        for (const auto& e : W[k]) {
            if (left[e.a].empty()) continue;
            auto& T = nl[e.c];
            if (T.empty()) T.assign(size_t(nd) * nd, 0.0);
            for (int i = 0; i < dl; ++i)
                for (int j = 0; j < dl; ++j) T[size_t(i * 4 + e.s) * nd + j * 4 + e.t] += left[e.a][size_t(i) * dl + j] * e.v;
        }
        left.swap(nl);
        dl = nd;
    }
    std::vector<std::vector<double>> right(bond_dim(L));
    right[idxF[L]] = {1.0};
    int dr = 1;
    for (int k = L - 1; k >= m; --k) {
        std::vector<std::vector<double>> nr(bond_dim(k));
        int nd = dr * 4;
        for (const auto& e : W[k]) {
            if (right[e.c].empty()) continue;
            auto& T = nr[e.a];
            if (T.empty()) T.assign(size_t(nd) * nd, 0.0);
            for (int i = 0; i < dr; ++i)
                for (int j = 0; j < dr; ++j) T[size_t(e.s * dr + i) * nd + e.t * dr + j] += e.v * right[e.c][size_t(i) * dr + j];
        }
        right.swap(nr);
        dr = nd;
    }
    size_t dim = size_t(dl) * dr;
    std::vector<double> H(dim * dim, 0.0);
    for (size_t w = 0; w < left.size(); ++w) {
        if (left[w].empty() || right[w].empty()) continue;
        for (int i = 0; i < dl; ++i)
            for (int j = 0; j < dl; ++j) {
                double a = left[w][size_t(i) * dl + j];
                if (a == 0.0) continue;
                for (int k = 0; k < dr; ++k)
                    for (int l = 0; l < dr; ++l)
                        H[(size_t(i) * dr + k) * dim + size_t(j) * dr + l] += a * right[w][size_t(k) * dr + l];
            }
    }
    return H;
}

}  // namespace gbd
