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

}  // namespace fdgb
