// schemes.cpp -- the SRJ scheme family on the host: App. B level table and the
// relaxation factors of Sec. 2, Eq. (srj-relaxation-parameters), in the order
// the sweeps apply them.
//
// For a cycle of length M:  lambda* solves T_M(lambda*) = 3, i.e.
//   lambda* = cosh(acosh(3) / M);
// the Chebyshev roots are x_j = cos((2j + 1) pi / (2M)), j = 0..M-1, and
//   omega_j = (lambda* + 1) / (2 (lambda* - x_j)).
// Application order within a cycle: Leja order of the roots on [-1, 1]
// starting from the largest root -- each next factor is the unused one whose
// root maximises the product of distances to the roots already used.  The
// paper (Sec. 2, last paragraph) asks only for an order that keeps roundoff
// and overflow under control; in exact arithmetic a cycle's effect does not
// depend on the order.
#include <cmath>
#include <vector>

#include "srj_internal.h"

namespace srj {

const int kLevelM[kNumLevels] = {1,   2,   3,   5,   7,   10,  14,   19,   26,
                                 35,  47,  63,  84,  111, 147, 194,  256,  338,
                                 446, 589, 778, 1027, 1356, 1790, 2362};

int level_offset(int level) {
    int off = 0;
    for (int l = 0; l < level; ++l) off += kLevelM[l];
    return off;
}

namespace {

// Factors of one level in application order.
std::vector<double> level_factors(int M) {
    const double lstar = std::cosh(std::acosh(3.0) / (double)M);
    std::vector<double> root(M), omega(M);
    for (int j = 0; j < M; ++j) {
        root[j] = std::cos((2.0 * j + 1.0) * M_PI / (2.0 * M));
        omega[j] = (lstar + 1.0) / (2.0 * (lstar - root[j]));
    }
    // Leja order: greedy maximisation of the log-distance sum.
    std::vector<double> logdist(M, 0.0);
    std::vector<bool> taken(M, false);
    std::vector<double> ordered;
    ordered.reserve(M);
    int pick = 0;
    while ((int)ordered.size() < M) {
        if (!ordered.empty()) {
            pick = -1;
            for (int j = 0; j < M; ++j)
                if (!taken[j] && (pick < 0 || logdist[j] > logdist[pick])) pick = j;
        }
        ordered.push_back(omega[pick]);
        taken[pick] = true;
        for (int j = 0; j < M; ++j)
            if (!taken[j]) logdist[j] += std::log(std::fabs(root[j] - root[pick]));
    }
    return ordered;
}

}  // namespace

void build_omega_table(double *out) {
    int off = 0;
    for (int l = 0; l < kNumLevels; ++l) {
        std::vector<double> w = level_factors(kLevelM[l]);
        for (int i = 0; i < kLevelM[l]; ++i) out[off + i] = w[i];
        off += kLevelM[l];
    }
}

int scheme_omegas(int level, double *out, int capacity) {
    if (level < 0 || level > kMaxLevel || out == nullptr) return -1;
    const int M = kLevelM[level];
    if (capacity < M) return -1;
    std::vector<double> w = level_factors(M);
    for (int i = 0; i < M; ++i) out[i] = w[i];
    return M;
}

}  // namespace srj
