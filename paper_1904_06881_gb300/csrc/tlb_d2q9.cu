// D2Q9 instantiation of the ternary ELBM kernels.
#include "tlb_kernels.cuh"
namespace tlb {
template struct Launch<2>;
template void ghosts_batch_launch<2>(const BatchEntry *, const int2 *, int, cudaStream_t);
}  // namespace tlb
