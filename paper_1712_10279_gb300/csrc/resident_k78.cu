// Instantiations of the resident kernels for K in {7, 8} channels (compiled apart
// from the other channel counts so that the units build in parallel).
#include "resident_kernel.cuh"

namespace vomt {
namespace res {

ResKernel res_kernel_k78(int K, int P, int NM, int LB, int LF)
{
    if (K == 7) return kernel_for<7>(P, NM, LB, LF);
    if (K == 8) return kernel_for<8>(P, NM, LB, LF);
    return nullptr;
}

MultiKernel res_multi_kernel_k78(int K, int P, int NM, int LB)
{
    if (K == 7) return multi_kernel_for<7>(P, NM, LB);
    if (K == 8) return multi_kernel_for<8>(P, NM, LB);
    return nullptr;
}

}  // namespace res
}  // namespace vomt
