// Problem set-up on the host: the diagonal D of the preconditioner (Sec. 7.1.1),
// the interval [t_min, t_max] of its spectrum (Sec. 4.3), a rigorous lower bound
// of the ground energy for the shift gamma (Sec. 3.1), alpha_0 and c of
// Cor. lrprecond, and the lowest determinants that start the subspace
// iteration (Sec. 7.1.4).  No device work.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.h"
#include "problem.h"

namespace bsm {
namespace {

// (spatial orbital, spin) of spin-orbital site i
inline void site_orbital(int i, int spin, int* p, int* s) {
    *p = spin ? i / 2 : i;
    *s = spin ? i % 2 : 0;
}

// v_ijkl = 1/2 (il|jk) of the spin-orbital Hamiltonian (Eq. (tvdef)); zero
// unless the spins of i, l and of j, k agree.
double v_so(const double* eri, int n, int spin, int i, int j, int k, int l) {
    int pi, si, pj, sj, pk, sk, pl, sl;
    site_orbital(i, spin, &pi, &si);
    site_orbital(j, spin, &pj, &sj);
    site_orbital(k, spin, &pk, &sk);
    site_orbital(l, spin, &pl, &sl);
    if (si != sl || sj != sk) return 0.0;
    return 0.5 * eri[(((size_t)pi * n + pl) * n + pj) * n + pk];
}

// Eigenvalues of a symmetric n x n matrix (row-major copy in a) by the cyclic
// Jacobi method: rotations annihilate a_pq until every off-diagonal entry is
// negligible against the diagonal.  Returned ascending.
std::vector<double> sym_eigenvalues(std::vector<double> a, int n) {
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += a[(size_t)p * n + p] * a[(size_t)p * n + p];
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        }
        if (off <= 1e-32 * diag || off == 0.0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
                // tan of the rotation angle: the smaller root of t^2 + 2 theta t - 1 = 0
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   // columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                a[(size_t)p * n + q] = a[(size_t)q * n + p] = 0.0;
            }
    }
    std::vector<double> ev(n);
    for (int p = 0; p < n; ++p) ev[p] = a[(size_t)p * n + p];
    std::sort(ev.begin(), ev.end());
    return ev;
}

}  // namespace

std::vector<double> precond_theta(int n_orb, const double* h, const double* eri, int spin, int n_particles,
                                  double gamma) {
    const int K = spin ? 2 * n_orb : n_orb;
    const int N = n_particles;
    std::vector<double> th(K);
    for (int i1 = 1; i1 <= K; ++i1) {
        const int i = i1 - 1;
        int p, s;
        site_orbital(i, spin, &p, &s);
        double acc = gamma / N + h[(size_t)p * n_orb + p];
        const int ki = std::max(0, i1 - N);
        for (int j1 = ki + 1; j1 <= ki + N; ++j1) {
            const int j = j1 - 1;
            acc += v_so(eri, n_orb, spin, i, j, j, i) - v_so(eri, n_orb, spin, i, j, i, j);
        }
        th[i] = acc;
    }
    return th;
}

void precond_interval(int n_orb, int spin, const double* theta, const double* h, int n_up, int n_dn, double* t_min,
                      double* t_max) {
    const int K = spin ? 2 * n_orb : n_orb;
    double lo = 0.0, hi = 0.0;
    const int ns = spin ? 2 : 1;
    for (int s = 0; s < ns; ++s) {
        const int n = s == 0 ? n_up : n_dn;
        if (n == 0) continue;
        std::vector<int> sites;
        for (int t = s; t < K; t += ns) sites.push_back(t);
        BSM_REQUIRE(n <= (int)sites.size(), BSMPS_ERR_CHARGE, "more particles than sites of a species");
        bool ordered = h != nullptr;
        for (size_t u = 0; ordered && u + 1 < sites.size(); ++u) {
            const int pa = spin ? sites[u] / 2 : sites[u], pb = spin ? sites[u + 1] / 2 : sites[u + 1];
            ordered = h[(size_t)pa * n_orb + pa] < h[(size_t)pb * n_orb + pb];
        }
        std::vector<double> vals;
        for (int t : sites) vals.push_back(theta[t]);
        if (!ordered) std::sort(vals.begin(), vals.end());
        for (int u = 0; u < n; ++u) lo += vals[u];
        for (int u = (int)vals.size() - n; u < (int)vals.size(); ++u) hi += vals[u];
    }
    *t_min = lo;
    *t_max = hi;
}

double energy_lower_bound(int n_orb, const double* h, const double* eri, int spin, int n_up, int n_dn,
                          int cholesky) {
    std::vector<double> a(h, h + (size_t)n_orb * n_orb);
    if (cholesky) {
        for (int p = 0; p < n_orb; ++p)
            for (int q = 0; q < n_orb; ++q) {
                double s = 0.0;
                for (int r = 0; r < n_orb; ++r) s += eri[(((size_t)p * n_orb + r) * n_orb + r) * n_orb + q];
                a[(size_t)p * n_orb + q] -= 0.5 * s;
            }
        for (int p = 0; p < n_orb; ++p)   // exact symmetry against rounding of the sums
            for (int q = p + 1; q < n_orb; ++q)
                a[(size_t)p * n_orb + q] = a[(size_t)q * n_orb + p] =
                    0.5 * (a[(size_t)p * n_orb + q] + a[(size_t)q * n_orb + p]);
    }
    const std::vector<double> ev = sym_eigenvalues(a, n_orb);
    double e = 0.0;
    for (int u = 0; u < n_up; ++u) e += ev[u];
    if (spin)
        for (int u = 0; u < n_dn; ++u) e += ev[u];
    return e;
}

// alpha_0 of Eq. (Sdef) and c of Eq. (precondcdef)
void precond_alpha0(double c0, double t_min, double c_lower, double c_upper, double* alpha0, double* c) {
    const double lo = c_lower * (1.0 - c0) * (1.0 - c0);
    const double hi = c_upper * (1.0 + c0) * (1.0 + c0);
    *alpha0 = std::sqrt(2.0 / (t_min * (lo + hi)));
    *c = (hi - lo) / (hi + lo);
}

// The D determinants of smallest sum_{i occupied} t_diag[i]; ties: occupation
// strings compared from site 0 with "occupied" first.  Enumerates the sector.
void lowest_determinants(int K, const double* t_diag, int spin, int n_up, int n_dn, int D, int64_t max_configs,
                         unsigned char* occ_out) {
    const int want[2] = {n_up, spin ? n_dn : 0};
    std::vector<int> pool[2];
    for (int i = 0; i < K; ++i) pool[spin ? i % 2 : 0].push_back(i);
    double total = 1.0;
    for (int s = 0; s < 2; ++s) {
        const int m = (int)pool[s].size(), k = want[s];
        BSM_REQUIRE(k >= 0 && k <= m, BSMPS_ERR_CHARGE, "more particles than sites of a species");
        double b = 1.0;
        for (int u = 0; u < k; ++u) b = b * (m - u) / (u + 1);
        total *= std::round(b);
    }
    BSM_REQUIRE(total <= (double)max_configs, BSMPS_ERR_RANK_CAP,
                "sector of " + std::to_string((long long)total) + " determinants is too large to enumerate");
    BSM_REQUIRE(total >= D, BSMPS_ERR_INVALID_ARG, "sector smaller than D");
    struct Row {
        double e;
        std::vector<unsigned char> occ;
    };
    std::vector<Row> rows;
    std::vector<int> ca, cb;
    // combinations of species 0 (outer) and species 1 (inner), lexicographic
    auto first = [](int k) {
        std::vector<int> c(k);
        for (int u = 0; u < k; ++u) c[u] = u;
        return c;
    };
    auto next = [](std::vector<int>& c, int m) {
        const int k = (int)c.size();
        int u = k - 1;
        while (u >= 0 && c[u] == m - k + u) --u;
        if (u < 0) return false;
        ++c[u];
        for (int v = u + 1; v < k; ++v) c[v] = c[v - 1] + 1;
        return true;
    };
    ca = first(want[0]);
    do {
        cb = first(want[1]);
        do {
            std::vector<unsigned char> occ(K, 0);
            for (int u : ca) occ[pool[0][u]] = 1;
            for (int u : cb) occ[pool[1][u]] = 1;
            double e = 0.0;
            for (int i = 0; i < K; ++i)
                if (occ[i]) e += t_diag[i];
            rows.push_back({e, std::move(occ)});
        } while (next(cb, (int)pool[1].size()));
    } while (next(ca, (int)pool[0].size()));
    std::stable_sort(rows.begin(), rows.end(), [](const Row& a, const Row& b) {
        if (a.e != b.e) return a.e < b.e;
        return a.occ > b.occ;   // occupied (1) before unoccupied (0) from site 0
    });
    for (int d = 0; d < D; ++d) std::memcpy(occ_out + (size_t)d * K, rows[d].occ.data(), K);
}

}  // namespace bsm
