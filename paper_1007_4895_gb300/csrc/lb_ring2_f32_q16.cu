/* Layout-10 step kernel (the ring-fed step as a persistent kernel over row queues) for
 * one storage format and one high-order set size (one translation unit each, so that
 * they compile in parallel). */
#include "lb_ring2.cuh"

namespace lbk {
template void launch_ring_units_store<1, 16>(const StepParams<float> &, const RingTab &, const RowQueues &,
                                              int, void *);
template int launch_ring_batch_store<1, 16>(const StepParams<float> *, const RingTab *, const uint32_t *,
                                                 const int2 *, const int *, int, int, int, int, unsigned int *, bool,
                                                 int, int *, void *);
}
