/*
 * lb_tma.h -- tensor maps for the TMA-fed step kernel (lb_step3.cu).
 *
 * One map per set and box shape over the 3-D storage of a time level:
 * (storage column, storage row, population plane) with extents (pitch, ny + 4, Q).
 */
#pragma once

#include <cuda.h>

#include "lb_internal.h"

struct TmaMaps {
    CUtensorMap box1[2];   /* per set: 136 columns x LB3_R rows x LB3_NP planes (a unit's rows) */
    CUtensorMap box2[2];   /* per set: 136 columns x (LB3_R + 4) rows x LB3_NP planes (plus the y halo) */
    CUtensorMap box5[2];   /* per set: 136 columns x (stream rows + 4) rows x 1 plane (streamed layout) */
};

namespace lbk {
int launch_step3(int store, const StepParams<float> &p, const TmaMaps &maps, int *err, void *stream);
int step3_rows();
int step3_cols();
int step3_planes();
/* Streamed layout (4): TMA-fed single-pass kernel on carried moments, with the wall,
 * ghost-row and mode-B work at the end of each unit (the pressure pass follows it).
 * FP32 / FP16 / BF16 storage. units: (tile, first row, rows,
 * set) runs of one set, at most stream_rows() rows, most work first; queue: a device
 * counter (reset by the launch). 0 on launch, -1 if unavailable. */
int launch_stream(int store, const StepParams<float> &p, const TmaMaps &maps, const int4 *units, int nunits,
                  unsigned int *queue, int *err, void *stream);
int stream_rows();   /* rows per work unit */
/* bounded-wait self-test: err (device int) gets `code` once the wait gives up */
int launch_wait_selftest(int *err, uint32_t polls, int code, void *stream);
int stream_cols();   /* columns per plane tile: 128 + 2 x 4 ghost */
}  // namespace lbk
