// Host-side helpers shared by the C-ABI translation units.
#pragma once

#include <stdint.h>

#include "fd.h"

// The grid handle behind fd_grid*.
struct fd_grid {
    int ndim;
    int64_t shape[3];
    double spacing[3];
    double origin[3];
};

namespace fdgb {

// Record a thread-local error message and return `status`.
fd_status set_error(fd_status status, const char *fmt, ...);

bool fornberg(int deriv, int n, const double *x, double z, double *weights_out);

// Layout of a field slot (fd_field_layout): rows of the contiguous axis
// padded to a multiple of 8 elements, no halo stored.
int64_t row_pitch(const fd_grid &g);
void layout_of(const fd_grid &g, int64_t *padded, int64_t *strides);

// Linear-interpolation table of npoint points (host FP64 coordinates
// [npoint][ndim]): base[p] is the slot-layout index of the lowest corner,
// weight[p * 8 + k] the FP32 weight of corner k.  One builder serves every
// sparse object and the allocation-free interpolation, so they agree by
// construction.  FD_ERR_OUT_OF_DOMAIN (message prefixed by `who`) for a
// point outside the grid.
fd_status linear_table(const fd_grid &g, int npoint, const double *coords, int64_t *base, float *weight,
                       const char *who);
// Offset of corner k from the lowest corner in the slot layout.
void corner_offsets(const fd_grid &g, int64_t off[8]);

}  // namespace fdgb
