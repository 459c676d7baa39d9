/* Step kernel instantiated for one storage format (kept in its own translation unit
 * so the formats compile in parallel). */
#include "lb_step_impl.cuh"

namespace lbk {
template void launch_step_store<4>(const StepParams<typename Store<4>::R> &, void *);
template void launch_step_desc_store<4>(const StepParams<typename Store<4>::R> &, int, void *);
template void launch_step_split_store<4>(const StepParams<typename Store<4>::R> &, int, const int2 *, int, void *, void *);
template int launch_batch_store<4>(const void *, const int *, int, int, int, int, unsigned int *, int, int, void *);
template int batch_blocks_per_sm<4>(int);
}
