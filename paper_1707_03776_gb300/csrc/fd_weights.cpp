// FD weights on the host in FP64 (fd_weights, fd_weights_central2).
//
// Fornberg's recurrence (B. Fornberg, "Generation of finite difference
// formulas on arbitrarily spaced grids", Math. Comp. 51, 1988) builds, node by
// node, the weights of every derivative order 0..deriv for the first j+1
// nodes from those for the first j nodes, without forming or solving the
// Vandermonde system.  The central second-derivative weights are that
// recurrence on the symmetric offsets -M..M.
#include <cmath>
#include <vector>

#include "fd_internal_host.h"

namespace fdgb {

// weights_out[j] = weight of f(x_j) in the derivative of order `deriv` at z.
// Returns false on repeated nodes.
bool fornberg(int deriv, int n, const double *x, double z, double *weights_out)
{
    // table[k][j]: weight of node j for derivative order k using the nodes seen so far
    std::vector<double> table((size_t)(deriv + 1) * n, 0.0);
    auto T = [&](int k, int j) -> double & { return table[(size_t)k * n + j]; };
    T(0, 0) = 1.0;
    double prod_prev = 1.0;       // prod_{l<i-1} (x_{i-1} - x_l)
    double dist_prev = x[0] - z;  // x_{i-1} - z
    for (int i = 1; i < n; i++) {
        int kmax = i < deriv ? i : deriv;
        double prod = 1.0;
        double dist = x[i] - z;
        for (int j = 0; j < i; j++) {
            double gap = x[i] - x[j];
            if (gap == 0.0) return false;
            prod *= gap;
            if (j == i - 1) {
                // the new node i, from the weights of node i-1 before its update
                for (int k = kmax; k >= 1; k--)
                    T(k, i) = prod_prev * (k * T(k - 1, i - 1) - dist_prev * T(k, i - 1)) / prod;
                T(0, i) = -prod_prev * dist_prev * T(0, i - 1) / prod;
            }
            // the old nodes j, folding in node i
            for (int k = kmax; k >= 1; k--) T(k, j) = (dist * T(k, j) - k * T(k - 1, j)) / gap;
            T(0, j) = dist * T(0, j) / gap;
        }
        prod_prev = prod;
        dist_prev = dist;
    }
    for (int j = 0; j < n; j++) weights_out[j] = T(deriv, j);
    return true;
}

}  // namespace fdgb

extern "C" fd_status fd_weights(int deriv, int n, const double *offsets, double *weights_out)
{
    using namespace fdgb;
    if (!offsets || !weights_out) return set_error(FD_ERR_INVALID_ARG, "fd_weights: null pointer");
    if (n < 1 || n > 64 || deriv < 0 || deriv >= n)
        return set_error(FD_ERR_INVALID_ARG, "fd_weights: need 0 <= deriv < n <= 64");
    for (int j = 0; j < n; j++)
        if (!std::isfinite(offsets[j])) return set_error(FD_ERR_INVALID_ARG, "fd_weights: non-finite offset");
    if (!fornberg(deriv, n, offsets, 0.0, weights_out))
        return set_error(FD_ERR_INVALID_ARG, "fd_weights: repeated offsets");
    return FD_OK;
}

extern "C" fd_status fd_weights_central2(int space_order, double *w_out)
{
    using namespace fdgb;
    if (!w_out) return set_error(FD_ERR_INVALID_ARG, "fd_weights_central2: null pointer");
    if (space_order < 2 || space_order > 16 || space_order % 2)
        return set_error(FD_ERR_UNSUPPORTED, "fd_weights_central2: space order must be even, 2..16");
    int M = space_order / 2;
    double x[17], w[17];
    for (int j = 0; j <= 2 * M; j++) x[j] = (double)(j - M);
    fornberg(2, 2 * M + 1, x, 0.0, w);
    for (int k = 0; k <= M; k++) w_out[k] = w[M + k];
    // enforce the exact symmetry of the central stencil (the recurrence is
    // symmetric only up to rounding) by averaging the mirrored weights
    for (int k = 1; k <= M; k++) w_out[k] = 0.5 * (w[M + k] + w[M - k]);
    return FD_OK;
}
