// rh.cu -- receding-horizon advance between two updates (Sec. 3.1, PI^2-RH):
// execute the first control of the new plan on the synthetic plant (one Euler
// step of the LWPR mean model at z = [x0, u_out[0]]) and warm-start the next
// update with the unexecuted remainder of the plan, the last control repeated.
#include "pi2rh_kernels.h"

namespace pi2rh {

namespace {

__global__ void rh_build_z(const float *__restrict__ x0, const float *__restrict__ u_out, float *z)
{
    const int c = threadIdx.x;
    if (c < NX) z[c] = x0[c];
    else if (c < NZ) z[c] = u_out[c - NX];
}

__global__ void rh_apply(float *__restrict__ x0, const float *__restrict__ y, float dt,
                         const float *__restrict__ u_out, int T, float *__restrict__ u_next)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NX && blockIdx.x == 0) x0[i] = fmaf(dt, y[i], x0[i]);
    if (i < T * NU) {
        const int t = i / NU, c = i % NU;
        const int src = t + 1 < T ? t + 1 : T - 1;
        u_next[i] = u_out[src * NU + c];
    }
}

}  // namespace

cudaError_t launch_rh_build_z(const float *x0, const float *u_out, float *z, cudaStream_t s)
{
    rh_build_z<<<1, 32, 0, s>>>(x0, u_out, z);
    return cudaGetLastError();
}

cudaError_t launch_rh_apply(float *x0, const float *y, float dt, const float *u_out, int T, float *u_next,
                            cudaStream_t s)
{
    const int n = T * NU > NX ? T * NU : NX;
    rh_apply<<<(n + 255) / 256, 256, 0, s>>>(x0, y, dt, u_out, T, u_next);
    return cudaGetLastError();
}

}  // namespace pi2rh
