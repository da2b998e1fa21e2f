// observables.h -- gap ratio, participation entropy and half-chain entanglement entropy.
#pragma once

#include "mbl_internal.h"

namespace mbl {

struct EntTables {
    int nblk = 0, dAmax = 0;
    std::vector<int32_t> dA;
    DVec<int32_t> d_idx, d_dA, d_dB;  // idx: ranks of a + b 2^{L/2}, block after block, row-major dA x dB
    DVec<int64_t> d_boff;
};

EntTables &ent_tables(Ctx *ctx, int L);
void observables_dev(Ctx *ctx, int L, int nev, const double *d_evals, const double *d_evecs, double *d_r,
                     double *d_rmean, double *d_s1p, double *d_se, cudaStream_t st);
// S^E of nev vectors (L <= 16, nev <= 64) on a static device scratch, no allocation (noalloc.cu)
void noalloc_setup(int device);
void entanglement_noalloc(Ctx *ctx, int L, int nev, const double *d_evecs, double *d_se, cudaStream_t st);

}  // namespace mbl
