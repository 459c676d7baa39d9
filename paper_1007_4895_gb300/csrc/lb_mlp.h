/*
 * lb_mlp.h -- internal interface between the learned-placement network (lb_mlp.cu) and
 * the lattice host code (lb_api.cu).
 */
#pragma once

#include <cstdint>
#include <string>

struct lb_mlp;

namespace lbk {
/* Inference with BF16 weights: x [8][n] raw features (device), p [n] (device), async. */
int mlp_infer_dev(lb_mlp *m, const float *x, int64_t n, float *p, void *stream);
/* message for lb_last_error() */
void set_last_error(const std::string &msg);
}  // namespace lbk
