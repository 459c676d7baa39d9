/* Layout-9 step kernel (paired FP32 arithmetic fed by a per-thread ring of asynchronous
 * copies) instantiated for one storage format (one translation unit per format so that
 * the formats compile in parallel). */
#include "lb_ring.cuh"

namespace lbk {
template void launch_ring_store<4>(const StepParams<float> &, void *);
}
