// D3Q27 instantiation of the ternary ELBM kernels.
#include "tlb_kernels.cuh"
namespace tlb {
template struct Launch<3>;
template void ghosts_batch_launch<3>(const BatchEntry *, const int2 *, int, cudaStream_t);
}  // namespace tlb
