// Host runtime internals: error reporting and weight/CFL helpers shared by
// the C-ABI implementation files.
#pragma once

#include <array>
#include <vector>

#include "../../include/fdwave.h"

namespace fdw {

// Record a thread-local message for fd_last_error() and return `code`.
int set_error(int code, const char *fmt, ...);
void clear_error();

// Orbit keys, multiplicities and weights of a stencil; optionally the full
// offset list (dz, dy, dx) with each offset's orbit index.
int compute_weights(const fd_stencil_desc *d, std::vector<std::array<int, 3>> &keys,
                    std::vector<int> &mult, std::vector<double> &w,
                    std::vector<std::array<int, 3>> *offsets, std::vector<int> *off_orbit);
int compute_cfl(const fd_stencil_desc *d, const std::vector<double> &w, double *cmax);

// fd_forward's body; `graphs` false launches the steps one by one on the
// caller's stream (no graph capture, instantiation or cache eviction).
int forward_impl(fd_plan *p, int model_kind, const float *model, int nsrc, const int64_t *src,
                 const float *wavelet, int nrec, const int64_t *rec, float *traces,
                 const float *state_in_d, float *state_out_d, void *ws, size_t ws_bytes,
                 void *stream, bool graphs);

}  // namespace fdw
