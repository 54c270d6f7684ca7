// nl_cg.cu -- conjugate gradients on -L x = f (placeholder until the solver lands).
#include "nl_internal.cuh"

nl_status nl_cg_release(nl_plan *p)
{
    if (p->cg_ws) cudaFree(p->cg_ws);
    if (p->cg_ws32) cudaFree(p->cg_ws32);
    if (p->cg_red) cudaFree(p->cg_red);
    if (p->cg_host) cudaFreeHost(p->cg_host);
    p->cg_ws = nullptr; p->cg_ws32 = nullptr; p->cg_red = nullptr; p->cg_host = nullptr;
    return NL_OK;
}

extern "C" nl_status nl_cg_solve(nl_plan *p, const void *f, void *x, int nrhs, double rtol,
                                 int maxit, int precond, nl_cg_stats *stats, void *stream)
{
    (void)f; (void)x; (void)nrhs; (void)rtol; (void)maxit; (void)precond; (void)stats; (void)stream;
    if (!nl_plan_ok(p)) {
        nl_set_error("nl_cg_solve: invalid plan");
        return NL_EINVAL;
    }
    nl_set_error("nl_cg_solve: not built yet");
    return NL_EUNSUPPORTED;
}
