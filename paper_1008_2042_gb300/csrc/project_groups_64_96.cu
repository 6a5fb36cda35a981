// Instantiations of the forward projector for column groups of 64, 80, 96 segments.
#include "project_kernel.cuh"

namespace cbct {

template const void *project_kernel<64>(int, int);
template const void *project_kernel<80>(int, int);
template const void *project_kernel<96>(int, int);

} // namespace cbct
