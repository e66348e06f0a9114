// Instantiations of the resident kernels for K in {3} channels (compiled apart
// from the other channel counts so that the units build in parallel).
#include "resident_kernel.cuh"

namespace vomt {
namespace res {

ResKernel res_kernel_k3(int K, int P, int NM, int LB, int LF)
{
    if (K == 3) return kernel_for<3>(P, NM, LB, LF);
    return nullptr;
}

MultiKernel res_multi_kernel_k3(int K, int P, int NM, int LB)
{
    if (K == 3) return multi_kernel_for<3>(P, NM, LB);
    return nullptr;
}

}  // namespace res
}  // namespace vomt
