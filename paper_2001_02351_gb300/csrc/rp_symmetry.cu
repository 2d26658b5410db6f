// Matrices at a reducible q from the irreducible one (Sec. 3.1, Eq. symeps): for a rotation S of the
// lattice with q* S = q + G_s, X_{G,G'}(q) = X_{G*,G'*}(q*) with G = G* S + G_s (no phase: the crystals
// here are symmorphic).  The host builds the index map; the kernel is a gather over all frequencies.
#include <algorithm>

#include "rp_internal.h"

namespace rp {

// X(q)[f][i][j] = X(q*)[f][perm[i]][perm[j]] (Sec. 3.1, Eq. symeps for a symmorphic crystal): one
// thread per output element, consecutive threads on consecutive j (coalesced writes, gathered reads)
__global__ void k_rotate(const double2* __restrict__ in, const int* __restrict__ perm, int n, long long total,
                         double2* __restrict__ out) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long nn = (long long)n * n;
        const long long f = e / nn, r = e % nn;
        const int i = (int)(r / n), j = (int)(r % n);
        out[e] = in[f * nn + (long long)perm[i] * n + perm[j]];
    }
}

cudaError_t launch_rotate(const double2* in, const int* perm, int n, int nf, double2* out, int num_sms,
                          cudaStream_t st) {
    const long long total = (long long)nf * n * n;
    const long long blocks = std::min<long long>((total + 255) / 256, (long long)num_sms * 16);
    k_rotate<<<(unsigned)std::max<long long>(1, blocks), 256, 0, st>>>(in, perm, n, total, out);
    return cudaGetLastError();
}

}  // namespace rp
