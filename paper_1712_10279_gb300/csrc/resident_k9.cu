// Instantiations of the resident kernel for K = 9 channels: the nine real
// coordinates of a complex Hermitian 3 x 3 field (complex matrix OMT), which runs
// with norms read at run time (NM = 0).  Compiled apart so that the units build in
// parallel.
#include "resident_kernel.cuh"

namespace vomt {
namespace res {

ResKernel res_kernel_k9(int K, int P, int NM, int LB, int LF)
{
    (void)LB;
    (void)LF;
    if (K != 9 || NM != 0) return nullptr;
    return P == 1 ? k_resident<9, 1, 0> : (P == 2 ? k_resident<9, 2, 0> : k_resident<9, 4, 0>);
}

}  // namespace res
}  // namespace vomt
