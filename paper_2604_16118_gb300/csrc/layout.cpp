// Charge-sector block index of block-sparse MPS (Sec. 2.3): sector sets,
// block dims of a fresh iterate, and the block layout of every core.
#include <algorithm>

#include "common.h"

namespace bsm {

int Bond::find(const Charge& c) const {
    auto it = std::lower_bound(q.begin(), q.end(), c);
    if (it == q.end() || !(*it == c)) return -1;
    return (int)(it - q.begin());
}

int Bond::total() const {
    int s = 0;
    for (int d : dim) s += d;
    return s;
}

std::vector<int> species_of(int n_orb, int spin) {
    std::vector<int> s;
    if (spin) {
        for (int p = 0; p < n_orb; ++p) {
            s.push_back(0);
            s.push_back(1);
        }
    } else {
        s.assign(n_orb, 0);
    }
    return s;
}

// Sets K_k of Sec. 2.3, generalised to two species: n_s in
// [max(0, N_s - R_s(b)), min(N_s, L_s(b))], ascending (n0, n1).
std::vector<std::vector<Charge>> valid_sectors(const std::vector<int>& species, Charge target) {
    int K = (int)species.size();
    int tot[2] = {0, 0};
    for (int s : species) tot[s]++;
    std::vector<std::vector<Charge>> out(K + 1);
    int L[2] = {0, 0};
    for (int b = 0; b <= K; ++b) {
        if (b > 0) L[species[b - 1]]++;
        int R0 = tot[0] - L[0], R1 = tot[1] - L[1];
        int lo0 = std::max(0, target.q0 - R0), hi0 = std::min(target.q0, L[0]);
        int lo1 = std::max(0, target.q1 - R1), hi1 = std::min(target.q1, L[1]);
        for (int a = lo0; a <= hi0; ++a)
            for (int c = lo1; c <= hi1; ++c) out[b].push_back({a, c});
    }
    return out;
}

static unsigned __int128 binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    unsigned __int128 r = 1;
    for (int i = 0; i < k; ++i) r = r * (unsigned)(n - i) / (unsigned)(i + 1);
    return r;
}

void Layout::rebuild_blocks() {
    blocks.assign(K, {});
    core_size.assign(K, 0);
    for (int t = 0; t < K; ++t) {
        int64_t off = 0;
        const Bond& bl = bonds[t];
        const Bond& br = bonds[t + 1];
        for (int li = 0; li < (int)bl.q.size(); ++li) {
            for (int sg = 0; sg < 2; ++sg) {
                int ri = br.find(bl.q[li] + site_delta(species[t], sg));
                if (ri < 0) continue;
                Block bk{li, ri, sg, bl.dim[li], br.dim[ri], off};
                off += (int64_t)bk.rows * bk.cols;
                blocks[t].push_back(bk);
            }
        }
        core_size[t] = off;
    }
}

int64_t Layout::total() const {
    int64_t s = 0;
    for (auto c : core_size) s += c;
    return s;
}

int Layout::block_index(int t, int li, int sigma) const {
    const auto& bl = blocks[t];
    for (int i = 0; i < (int)bl.size(); ++i)
        if (bl[i].li == li && bl[i].sigma == sigma) return i;
    return -1;
}

void check_layout(const Layout& L) {
    BSM_REQUIRE((int)L.bonds.size() == L.K + 1, BSMPS_ERR_INVALID_ARG, "bond count != K+1");
    auto valid = valid_sectors(L.species, L.target);
    for (int b = 0; b <= L.K; ++b) {
        const Bond& bd = L.bonds[b];
        for (size_t i = 0; i < bd.q.size(); ++i) {
            BSM_REQUIRE(bd.dim[i] > 0, BSMPS_ERR_INVALID_ARG, "sector of dimension <= 0");
            BSM_REQUIRE(i == 0 || bd.q[i - 1] < bd.q[i], BSMPS_ERR_INVALID_ARG,
                        "sectors of a bond must be strictly ascending");
            BSM_REQUIRE(std::find(valid[b].begin(), valid[b].end(), bd.q[i]) != valid[b].end(),
                        BSMPS_ERR_CHARGE, "sector not realisable for the target particle numbers");
        }
    }
    if (!L.bonds[0].q.empty()) {
        BSM_REQUIRE(L.bonds[0].q.size() == 1 && L.bonds[0].dim[0] == 1, BSMPS_ERR_INVALID_ARG,
                    "bond 0 must be the single sector (0,0) of dim 1");
    }
    if (!L.bonds[L.K].q.empty()) {
        // dim > 1: the column index of a joint block MPS (Sec. 6.2)
        BSM_REQUIRE(L.bonds[L.K].q.size() == 1, BSMPS_ERR_INVALID_ARG,
                    "bond K must be the single target sector");
    }
}

// Block dims of a fresh iterate (see bsmps_mps_random_size).
Layout default_layout(const std::vector<int>& species, Charge target, int r_max, int D) {
    Layout L;
    L.K = (int)species.size();
    L.species = species;
    L.target = target;
    int tot[2] = {0, 0};
    for (int s : species) tot[s]++;
    BSM_REQUIRE(target.q0 >= 0 && target.q1 >= 0 && target.q0 <= tot[0] && target.q1 <= tot[1],
                BSMPS_ERR_CHARGE, "particle numbers exceed the number of sites");
    auto valid = valid_sectors(species, target);
    int Lc[2] = {0, 0};
    L.bonds.resize(L.K + 1);
    for (int b = 0; b <= L.K; ++b) {
        if (b > 0) Lc[species[b - 1]]++;
        int R0 = tot[0] - Lc[0], R1 = tot[1] - Lc[1];
        std::vector<unsigned __int128> lc, rc;
        unsigned __int128 exact_sum = 0, wsum = 0;
        for (const Charge& q : valid[b]) {
            unsigned __int128 l = binom(Lc[0], q.q0) * binom(Lc[1], q.q1);
            unsigned __int128 r = binom(R0, target.q0 - q.q0) * binom(R1, target.q1 - q.q1) * (unsigned)D;
            lc.push_back(l);
            rc.push_back(r);
            exact_sum += std::min(l, r);
            wsum += l * r;
        }
        for (size_t i = 0; i < valid[b].size(); ++i) {
            unsigned __int128 d;
            if (exact_sum <= (unsigned __int128)r_max) {
                d = std::min(lc[i], rc[i]);
            } else {
                unsigned __int128 prop = ((unsigned __int128)r_max * lc[i] * rc[i]) / wsum;
                d = std::min(std::min(lc[i], rc[i]), prop);
            }
            if (d > 0) {
                L.bonds[b].q.push_back(valid[b][i]);
                L.bonds[b].dim.push_back((int)d);
            }
        }
    }
    L.rebuild_blocks();
    return L;
}

// Rank-one e_1 (Sec. 7.1.4): first n_up species-0 and n_dn species-1 sites occupied.
Layout e1_layout(const std::vector<int>& species, Charge target) {
    Layout L;
    L.K = (int)species.size();
    L.species = species;
    L.target = target;
    L.bonds.resize(L.K + 1);
    Charge q{0, 0};
    int seen[2] = {0, 0};
    L.bonds[0].q.push_back(q);
    L.bonds[0].dim.push_back(1);
    for (int t = 0; t < L.K; ++t) {
        int s = species[t];
        int want = s == 0 ? target.q0 : target.q1;
        int o = seen[s] < want ? 1 : 0;
        seen[s] += o;
        q = q + site_delta(s, o);
        L.bonds[t + 1].q.push_back(q);
        L.bonds[t + 1].dim.push_back(1);
    }
    BSM_REQUIRE(q == target, BSMPS_ERR_CHARGE, "particle numbers exceed the number of sites");
    L.rebuild_blocks();
    return L;
}

Layout determinant_layout(const std::vector<int>& species, Charge target, const unsigned char* occ, int D,
                          std::vector<double>* values) {
    const int K = (int)species.size();
    BSM_REQUIRE(D >= 1 && occ, BSMPS_ERR_INVALID_ARG, "D >= 1 occupation strings required");
    // charge path and index of every vector on every bond
    std::vector<std::vector<Charge>> path(D, std::vector<Charge>(K + 1));
    for (int i = 0; i < D; ++i) {
        Charge q{0, 0};
        path[i][0] = q;
        for (int t = 0; t < K; ++t) {
            const unsigned char o = occ[(size_t)i * K + t];
            BSM_REQUIRE(o <= 1, BSMPS_ERR_INVALID_ARG, "occupations must be 0 or 1");
            q = q + site_delta(species[t], o);
            path[i][t + 1] = q;
        }
        BSM_REQUIRE(q == target, BSMPS_ERR_CHARGE, "occupation string outside the particle sector");
    }
    Layout L;
    L.K = K;
    L.species = species;
    L.target = target;
    L.bonds.resize(K + 1);
    std::vector<std::vector<int>> pos(D, std::vector<int>(K + 1, 0));
    for (int b = 0; b <= K; ++b) {
        std::vector<Charge> qs;
        for (int i = 0; i < D; ++i) qs.push_back(path[i][b]);
        std::sort(qs.begin(), qs.end());
        qs.erase(std::unique(qs.begin(), qs.end()), qs.end());
        std::vector<int> cnt(qs.size(), 0);
        for (int i = 0; i < D; ++i) {
            const int s = (int)(std::lower_bound(qs.begin(), qs.end(), path[i][b]) - qs.begin());
            if (b == 0) {
                cnt[s] = 1;
                pos[i][b] = 0;
            } else if (b == K) {
                cnt[s] = D;
                pos[i][b] = i;
            } else {
                pos[i][b] = cnt[s]++;
            }
        }
        L.bonds[b].q = qs;
        L.bonds[b].dim = cnt;
    }
    L.rebuild_blocks();
    values->assign((size_t)L.total(), 0.0);
    int64_t base = 0;
    for (int t = 0; t < K; ++t) {
        for (int i = 0; i < D; ++i) {
            const int li = L.bonds[t].find(path[i][t]);
            const int bi = L.block_index(t, li, occ[(size_t)i * K + t]);
            const Block& bk = L.blocks[t][bi];
            (*values)[(size_t)(base + bk.off + (int64_t)pos[i][t] * bk.cols + pos[i][t + 1])] = 1.0;
        }
        base += L.core_size[t];
    }
    return L;
}

}  // namespace bsm
