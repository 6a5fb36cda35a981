// Instantiations of the forward projector for column groups of 16, 24, 32 segments.
#include "project_kernel.cuh"

namespace cbct {

template const void *project_kernel<16>(int, int);
template const void *project_kernel<24>(int, int);
template const void *project_kernel<32>(int, int);

} // namespace cbct
