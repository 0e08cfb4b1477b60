// D3Q27 instantiation of the ternary ELBM kernels.
#include "tlb_kernels.cuh"
namespace tlb {
template struct Launch<3>;
}  // namespace tlb
