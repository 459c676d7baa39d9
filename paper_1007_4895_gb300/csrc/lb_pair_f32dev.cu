/* Layout-7 step kernel (paired FP32 arithmetic) instantiated for one storage format
 * (kept in its own translation unit so the formats compile in parallel). */
#include "lb_pair.cuh"

namespace lbk {
template void launch_pair_store<2>(const StepParams<float> &, void *);

size_t pair_table_bytes() { return sizeof(PairTables); }

void launch_pair_table(const StepParams<float> &p, void *dst, void *stream)
{
    pair_table_kernel<<<1, 128, 0, static_cast<cudaStream_t>(stream)>>>(p, static_cast<PairTables *>(dst));
}
}
