// nf_adjoint.cu -- discrete adjoint of the RK4 map (placeholder until the adjoint
// pair kernel lands).
#include "nf_internal.cuh"

using namespace nfi;

extern "C" nf_status nf_adjoint(nf_operator *op, const float *ckpt, int C, int B, double t0, double dt, int nsteps,
                                const float *beta, const float *theta, const nf_forcing *g, const float *lambda_T,
                                float *grad_u0, float *grad_kernel, void *stream) {
    clear_error();
    return fail(NF_ERR_UNSUPPORTED, "nf_adjoint is not built yet");
}
