// Exact MPO of the second-quantized Hamiltonian H_gamma (Sec. 2.4, Eq. (hamil),
// Thm. opranks), built as a finite-state operator from canonicalised
// Jordan--Wigner terms:
//  * a term coef * prod a^(*) equals coef * (x)_t L_t with site-local 2x2
//    factors (A, A^T at the operators' own sites, Z left of them, I right);
//  * the sites a term touches, with their factors normalised to a leading +1,
//    form its canonical key; terms with equal keys are merged;
//  * the channel of a term at bond b is I (nothing placed), F (all placed),
//    the placed prefix (fewer placed than remaining, or equal and b < K/2) or
//    the remaining suffix; the coefficient rides on the single transition
//    from {I, prefix} to {suffix, F}; idle sites carry Z^(channel parity).
#include <algorithm>
#include <cmath>
#include <unordered_map>
#include <unordered_set>

#include "common.h"

namespace bsm {
namespace {

struct M2 {
    long long m[2][2];
};

const M2 kI = {{{1, 0}, {0, 1}}};
const M2 kZ = {{{1, 0}, {0, -1}}};
const M2 kA = {{{0, 1}, {0, 0}}};    // annihilation: |1> -> |0>
const M2 kAT = {{{0, 0}, {1, 0}}};   // creation

M2 mul(const M2& x, const M2& y) {
    M2 r{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) r.m[i][j] = x.m[i][0] * y.m[0][j] + x.m[i][1] * y.m[1][j];
    return r;
}

int code_of(const M2& x) {
    int c = 0, p = 1;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            c += (int)(x.m[i][j] + 1) * p;
            p *= 3;
        }
    return c;
}

M2 from_code(int c) {
    M2 r{};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            r.m[i][j] = c % 3 - 1;
            c /= 3;
        }
    return r;
}

bool code_odd(int c) {
    M2 r = from_code(c);
    return r.m[0][1] != 0 || r.m[1][0] != 0;
}

int code_charge(int c) {
    M2 r = from_code(c);
    if (r.m[1][0] != 0) return 1;
    if (r.m[0][1] != 0) return -1;
    return 0;
}

// A canonical key packs up to four (site, code) pairs, first pair most
// significant, each as site*128 + code + 1 in 16 bits (0 = absent), so that
// integer order equals lexicographic order with shorter prefixes first.
constexpr int kMaxOps = 4;

inline uint64_t pair_val(int site, int code) { return (uint64_t)(site * 128 + code + 1); }
inline int key_len(uint64_t k) {
    int n = 0;
    for (int i = 0; i < kMaxOps; ++i)
        if ((k >> (16 * (kMaxOps - 1 - i))) & 0xffff) n++;
    return n;
}
inline int key_site(uint64_t k, int i) {
    return (int)(((k >> (16 * (kMaxOps - 1 - i))) & 0xffff) - 1) / 128;
}
inline int key_code(uint64_t k, int i) {
    return (int)(((k >> (16 * (kMaxOps - 1 - i))) & 0xffff) - 1) % 128;
}
inline uint64_t key_slice(uint64_t k, int from, int to) {   // pairs [from, to) re-based
    uint64_t r = 0;
    for (int i = from; i < to; ++i) {
        uint64_t v = (k >> (16 * (kMaxOps - 1 - i))) & 0xffff;
        r |= v << (16 * (kMaxOps - 1 - (i - from)));
    }
    return r;
}

// Canonical key of coef * prod(ops); returns false when the product vanishes.
bool canonical(const int* sites, const bool* cr, int nops, uint64_t* key, int* sign) {
    int us[kMaxOps];
    int nu = 0;
    for (int i = 0; i < nops; ++i) us[nu++] = sites[i];
    std::sort(us, us + nu);
    nu = (int)(std::unique(us, us + nu) - us);
    uint64_t k = 0;
    int sg = 1;
    for (int u = 0; u < nu; ++u) {
        int t = us[u];
        M2 M = kI;
        for (int i = 0; i < nops; ++i) {
            const M2& f = sites[i] == t ? (cr[i] ? kAT : kA) : (sites[i] > t ? kZ : kI);
            M = mul(M, f);
        }
        long long first = 0;
        for (int i = 0; i < 2 && !first; ++i)
            for (int j = 0; j < 2 && !first; ++j)
                if (M.m[i][j] != 0) first = M.m[i][j];
        if (!first) return false;
        if (first < 0) {
            for (auto& row : M.m)
                for (auto& v : row) v = -v;
            sg = -sg;
        }
        k |= pair_val(t, code_of(M)) << (16 * (kMaxOps - 1 - u));
    }
    *key = k;
    *sign = sg;
    return true;
}

// Channel state: kind 0 = I, 1 = prefix, 2 = suffix, 3 = F.
struct State {
    int kind;
    uint64_t ops;
    int len;
    bool operator==(const State& o) const {
        return kind == o.kind && ops == o.ops && len == o.len;
    }
    bool operator<(const State& o) const {
        if (kind != o.kind) return kind < o.kind;
        if (len != o.len) return len < o.len;
        return ops < o.ops;
    }
};

struct StateHash {
    size_t operator()(const State& s) const {
        return std::hash<uint64_t>()(s.ops * 1000003ull + (uint64_t)s.kind * 31 + s.len);
    }
};

State state_of(uint64_t key, int m, int b, int bmid) {
    int p = 0;
    for (int i = 0; i < m; ++i)
        if (key_site(key, i) < b) p++;
    if (p == 0) return {0, 0, 0};
    if (p == m) return {3, 0, 0};
    if (p < m - p || (p == m - p && b < bmid)) return {1, key_slice(key, 0, p), p};
    return {2, key_slice(key, p, m), m - p};
}

int parity(const State& s) {
    if (s.kind == 0 || s.kind == 3) return 0;
    int par = 0;
    for (int i = 0; i < s.len; ++i) par ^= code_odd(key_code(s.ops, i)) ? 1 : 0;
    return par;
}

struct WCell {
    double v[2][2];
    bool mask[2][2];
};

}  // namespace

Mpo build_mpo(int n_orb, const double* h, const double* eri, int spin, int n_particles,
              double gamma, double compress_tol) {
    BSM_REQUIRE(n_orb > 0 && h != nullptr && eri != nullptr, BSMPS_ERR_INVALID_ARG,
                "mpo_from_integrals: n_orb > 0 and non-null h, eri required");
    const int n = n_orb;
    const int nspin = spin ? 2 : 1;
    auto so = [&](int p, int s) { return spin ? 2 * p + s : p; };
    const double shift = n_particles > 0 ? gamma / n_particles : 0.0;

    // 1. canonical terms, merged in enumeration order (Eq. (hamil), (tvdef))
    std::unordered_map<uint64_t, double> acc;
    acc.reserve(1 << 16);
    auto add_term = [&](double coef, const int* sites, const bool* cr, int nops) {
        uint64_t key;
        int sg;
        if (!canonical(sites, cr, nops, &key, &sg)) return;
        acc[key] += sg * coef;
    };
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double coef = h[p * n + q] + (p == q ? shift : 0.0);
            if (coef == 0.0) continue;
            for (int s = 0; s < nspin; ++s) {
                int st[2] = {so(p, s), so(q, s)};
                bool cr[2] = {true, false};
                add_term(coef, st, cr, 2);
            }
        }
    const size_t n2 = (size_t)n * n, n3 = n2 * n;
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) {
                    double e = eri[p * n3 + q * n2 + r * (size_t)n + s];
                    if (e == 0.0) continue;
                    double val = 0.5 * e;
                    for (int sa = 0; sa < nspin; ++sa)
                        for (int sb = 0; sb < nspin; ++sb) {
                            // v_ijkl a_i^* a_j^* a_k a_l with i=p, j=r, k=s, l=q
                            int st[4] = {so(p, sa), so(r, sb), so(s, sb), so(q, sa)};
                            bool cr[4] = {true, true, false, false};
                            add_term(val, st, cr, 4);
                        }
                }
    std::vector<std::pair<uint64_t, double>> terms;
    terms.reserve(acc.size());
    for (auto& kv : acc)
        if (kv.second != 0.0 && std::fabs(kv.second) > compress_tol) terms.push_back(kv);
    std::sort(terms.begin(), terms.end(),
              [](const std::pair<uint64_t, double>& x, const std::pair<uint64_t, double>& y) {
                  return x.first < y.first;
              });

    const std::vector<int> species = species_of(n_orb, spin);
    const int K = (int)species.size();
    const int bmid = K / 2;

    // 2. channels per bond
    std::vector<std::unordered_set<State, StateHash>> sets(K + 1);
    for (int b = 0; b < K; ++b) sets[b].insert({0, 0, 0});
    for (int b = 1; b <= K; ++b) sets[b].insert({3, 0, 0});
    for (auto& tm : terms) {
        uint64_t key = tm.first;
        int m = key_len(key);
        int s1 = key_site(key, 0), sm = key_site(key, m - 1);
        for (int b = s1 + 1; b <= sm; ++b) sets[b].insert(state_of(key, m, b, bmid));
    }
    std::vector<std::vector<State>> chans(K + 1);
    std::vector<std::unordered_map<State, int, StateHash>> index(K + 1);
    Mpo W;
    W.K = K;
    W.species = species;
    W.charges.resize(K + 1);
    for (int b = 0; b <= K; ++b) {
        chans[b].assign(sets[b].begin(), sets[b].end());
        std::sort(chans[b].begin(), chans[b].end());
        for (int i = 0; i < (int)chans[b].size(); ++i) {
            const State& st = chans[b][i];
            index[b][st] = i;
            Charge d{0, 0};
            for (int j = 0; j < st.len; ++j) {
                int c = code_charge(key_code(st.ops, j));
                Charge dd = site_delta(species[key_site(st.ops, j)], 1);
                if (st.kind == 1) {
                    d.q0 += c * dd.q0;
                    d.q1 += c * dd.q1;
                } else if (st.kind == 2) {
                    d.q0 -= c * dd.q0;
                    d.q1 -= c * dd.q1;
                }
            }
            W.charges[b].push_back(d);
        }
    }

    // 3. operator-valued cores
    std::vector<std::unordered_map<uint64_t, WCell>> cells(K);
    auto put = [&](int t, int a, int b, const M2& M, double weight, bool accumulate) {
        uint64_t ck = ((uint64_t)a << 32) | (uint32_t)b;
        auto it = cells[t].find(ck);
        if (it == cells[t].end()) {
            WCell c;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    c.v[i][j] = weight * (double)M.m[i][j];
                    c.mask[i][j] = M.m[i][j] != 0;
                }
            cells[t].emplace(ck, c);
        } else {
            WCell& c = it->second;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    if (accumulate) c.v[i][j] = c.v[i][j] + weight * (double)M.m[i][j];
                    c.mask[i][j] = c.mask[i][j] || M.m[i][j] != 0;
                }
        }
    };
    const State sI{0, 0, 0}, sF{3, 0, 0};
    W.ident_last = index[K - 1][sI];
    for (int t = 0; t + 1 < K; ++t) put(t, index[t][sI], index[t + 1][sI], kI, 1.0, false);
    for (int t = 1; t < K; ++t) put(t, index[t][sF], index[t + 1][sF], kI, 1.0, false);
    {
        int fb = index[1][sF];
        WCell c{};
        c.mask[0][0] = c.mask[1][1] = true;
        cells[0][((uint64_t)0 << 32) | (uint32_t)fb] = c;
    }
    for (auto& tm : terms) {
        uint64_t key = tm.first;
        double coef = tm.second;
        int m = key_len(key);
        int s1 = key_site(key, 0), sm = key_site(key, m - 1);
        int pos = 0;
        for (int t = s1; t <= sm; ++t) {
            State prev = state_of(key, m, t, bmid);
            State nxt = state_of(key, m, t + 1, bmid);
            int a = index[t][prev];
            int b = index[t + 1][nxt];
            M2 M;
            if (pos < m && key_site(key, pos) == t) {
                M = from_code(key_code(key, pos));
                pos++;
            } else {
                M = parity(prev) ? kZ : kI;
            }
            bool is_coef = (prev.kind == 0 || prev.kind == 1) && (nxt.kind == 2 || nxt.kind == 3);
            put(t, a, b, M, is_coef ? coef : 1.0, is_coef);
        }
    }
    W.entries.resize(K);
    for (int t = 0; t < K; ++t) {
        std::vector<std::pair<uint64_t, WCell>> cv(cells[t].begin(), cells[t].end());
        std::sort(cv.begin(), cv.end(),
                  [](const std::pair<uint64_t, WCell>& x, const std::pair<uint64_t, WCell>& y) {
                      return x.first < y.first;
                  });
        for (auto& kv : cv) {
            int a = (int)(kv.first >> 32), b = (int)(kv.first & 0xffffffffu);
            for (int so_ = 0; so_ < 2; ++so_)
                for (int si = 0; si < 2; ++si)
                    if (kv.second.mask[so_][si]) {
                        if (t == 0 && a == 0 && b == W.bond_dim(1) - 1 && so_ == si)
                            W.shift_entry[so_] = (int)W.entries[0].size();
                        W.entries[t].push_back({a, b, so_, si, kv.second.v[so_][si]});
                    }
        }
    }
    return W;
}

}  // namespace bsm
