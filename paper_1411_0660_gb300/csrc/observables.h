// observables.h -- eigenvector observables: gap ratio, participation entropies, half-chain
// entanglement entropy, KL divergence of adjacent eigenvectors, bipartite fluctuation, dynamic fraction.
#pragma once

#include "mbl_internal.h"

namespace mbl {

struct EntTables {
    int nblk = 0, dAmax = 0;
    std::vector<int32_t> dA;
    DVec<int32_t> d_idx, d_dA, d_dB;  // idx: ranks of a + b 2^{floor(L/2)}, block after block, row-major dA x dB
    DVec<int64_t> d_boff;
    DVec<uint32_t> d_states;  // the sector's basis states in ascending order
    // per basis state: S^z of the half chain A and M = sum_j S^z_j e^{2 pi i j / L} (re, im)
    DVec<double> d_mA, d_Mre, d_Mim;
    // scratch of observables_extra_dev (partial sums, squared norms), grown on demand
    DVec<double> x_part, x_nrm;
    size_t x_part_cap = 0, x_nrm_cap = 0;
};

// tables of the sector (L, nup): Schmidt blocks of the cut after site floor(L/2) - 1, per-state S^z_A and M
EntTables &ent_tables(Ctx *ctx, int L, int nup);
void observables_dev(Ctx *ctx, int L, int nup, int nev, const double *d_evals, const double *d_evecs, double *d_r,
                     double *d_rmean, double *d_s1p, double *d_se, cudaStream_t st);
// KL of adjacent vectors (nev - 1), S_q^P, bipartite fluctuation F and dynamic fraction f (nev each),
// enqueued on st (no synchronization; scratch from the per-L cache)
void observables_extra_dev(Ctx *ctx, int L, int nup, int nev, const double *d_evecs, double q, double *d_kl,
                           double *d_sqp, double *d_fluct, double *d_dynf, cudaStream_t st);
// S^E of nev vectors (L <= 16, nev <= 64) on a static device scratch, no allocation (noalloc.cu)
void noalloc_setup(int device);
void entanglement_noalloc(Ctx *ctx, int L, int nev, const double *d_evecs, double *d_se, cudaStream_t st);

}  // namespace mbl
