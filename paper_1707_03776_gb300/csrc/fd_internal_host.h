// Host-side helpers shared by the C-ABI translation units.
#pragma once

#include "fd.h"

namespace fdgb {

// Record a thread-local error message and return `status`.
fd_status set_error(fd_status status, const char *fmt, ...);

bool fornberg(int deriv, int n, const double *x, double z, double *weights_out);

}  // namespace fdgb
