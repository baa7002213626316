// mpo.h -- left/right operator sets of Eq. 1 at every cut (host tables; the term
// split of Sec. II.B step 1).
#pragma once

#include <cstdint>
#include <vector>

#include "core.h"

namespace gbd {

// One nonzero of W[k]: state a at cut k -> state c at cut k+1, local matrix
// element <s| . |t> of the orbital-k factor.
struct MpoEntry {
    int a, c;
    int s, t;
    double v;
};

struct Mpo {
    int L = 0;
    int ksw = 0;                            // first cut with complementary pairs
    std::vector<std::vector<Q>> dq;         // per cut, per state: left-part change
    std::vector<std::vector<MpoEntry>> W;   // per site
    std::vector<int> idxI, idxF;            // per cut: index of the I / F state or -1

    // Eq. 1 with chemist integrals; see mpo.cpp for the construction.
    void build(int L, const double* h, const double* eri, int ksw);
    int bond_dim(int cut) const { return int(dq[cut].size()); }
    // Dense 4^L x 4^L contraction (L <= 5), for host-side checks.
    std::vector<double> dense() const;
};

}  // namespace gbd
