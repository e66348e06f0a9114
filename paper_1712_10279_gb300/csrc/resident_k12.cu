// Instantiations of the resident kernels for K in {1, 2} channels (compiled apart
// from the other channel counts so that the units build in parallel).
#include "resident_kernel.cuh"

namespace vomt {
namespace res {

ResKernel res_kernel_k12(int K, int P, int NM, int LB, int LF)
{
    if (K == 1) return kernel_for<1>(P, NM, LB, LF);
    if (K == 2) return kernel_for<2>(P, NM, LB, LF);
    return nullptr;
}

MultiKernel res_multi_kernel_k12(int K, int P, int NM, int LB)
{
    if (K == 1) return multi_kernel_for<1>(P, NM, LB);
    if (K == 2) return multi_kernel_for<2>(P, NM, LB);
    return nullptr;
}

}  // namespace res
}  // namespace vomt
