// Instantiations of the forward projector for column groups of 40, 48, 56 segments.
#include "project_kernel.cuh"

namespace cbct {

template const void *project_kernel<40>(int, int);
template const void *project_kernel<48>(int, int);
template const void *project_kernel<56>(int, int);

} // namespace cbct
