// ism_batched.cu -- ensemble of independent pressure solves.
#include "ism_internal.cuh"

extern "C" ism_status ism_solve_batched(int n, ism_ctx *const *ctxs, const double *const *rhs,
                                        double *const *p, double tol, int max_cycles,
                                        int *cycles_out, double *relres_out)
{
    if (n < 0 || (n > 0 && (!ctxs || !rhs || !p)) || !(tol > 0.0) || max_cycles < 0) return ISM_ERR_ARG;
    ism_status first = ISM_OK;
    for (int k = 0; k < n; ++k) {
        int c = 0;
        double r = 0.0;
        ism_status s = ism_solve(ctxs[k], rhs[k], p[k], tol, max_cycles, &c, &r);
        if (cycles_out) cycles_out[k] = c;
        if (relres_out) relres_out[k] = r;
        if (s != ISM_OK && first == ISM_OK) first = s;
    }
    return first;
}
