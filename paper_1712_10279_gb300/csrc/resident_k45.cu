// Instantiations of the resident kernels for K in {4, 5} channels (compiled apart
// from the other channel counts so that the units build in parallel).
#include "resident_kernel.cuh"

namespace vomt {
namespace res {

ResKernel res_kernel_k45(int K, int P, int NM, int LB, int LF)
{
    if (K == 4) return kernel_for<4>(P, NM, LB, LF);
    if (K == 5) return kernel_for<5>(P, NM, LB, LF);
    return nullptr;
}

MultiKernel res_multi_kernel_k45(int K, int P, int NM, int LB)
{
    if (K == 4) return multi_kernel_for<4>(P, NM, LB);
    if (K == 5) return multi_kernel_for<5>(P, NM, LB);
    return nullptr;
}

}  // namespace res
}  // namespace vomt
