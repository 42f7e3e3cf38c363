// Solvers around the grouped transform: LSQR (Sec. 4.1) and FISTA (Sec. 4.2).
#include "internal.cuh"

extern "C" {

int lsqr_solve(anova_plan_t plan, const void *y_dev, const double *w_dev, double lambda, int max_it, double atol,
               double btol, void *fhat_dev, anova_solve_info *info) {
    (void)plan; (void)y_dev; (void)w_dev; (void)lambda; (void)max_it; (void)atol; (void)btol; (void)fhat_dev;
    (void)info;
    return ANOVA_ERR_UNSUPPORTED;
}

int fista_solve(anova_plan_t plan, const void *y_dev, const double *w_dev, const double *lambdas, int n_lambda,
                int max_it, double tol, int step_mode, double L0, double eta, const uint8_t *group_mask,
                int warm_start, void *fhat_path_dev, anova_solve_info *info) {
    (void)plan; (void)y_dev; (void)w_dev; (void)lambdas; (void)n_lambda; (void)max_it; (void)tol; (void)step_mode;
    (void)L0; (void)eta; (void)group_mask; (void)warm_start; (void)fhat_path_dev; (void)info;
    return ANOVA_ERR_UNSUPPORTED;
}

}  // extern "C"
