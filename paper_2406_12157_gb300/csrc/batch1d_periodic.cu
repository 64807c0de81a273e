// batch1d_periodic.cu -- the periodic instantiations of the persistent batch
// kernel (a translation unit of its own so that the two boundary variants
// compile in parallel).
#include "batch1d_kernel.cuh"

namespace she {

void* batch_kernel_periodic(bool species)
{
    return species ? (void*)k_step1d_batch<false, true> : (void*)k_step1d_batch<false, false>;
}

}  // namespace she
