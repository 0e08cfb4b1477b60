// D2Q9 instantiation of the ternary ELBM kernels.
#include "tlb_kernels.cuh"
namespace tlb {
template struct Launch<2>;
}  // namespace tlb
