/* Layout-7 step kernel (paired FP32 arithmetic) instantiated for one storage format
 * (kept in its own translation unit so the formats compile in parallel). */
#include "lb_pair.cuh"

namespace lbk {
template void launch_pair_store<1>(const StepParams<float> &, void *);
}
