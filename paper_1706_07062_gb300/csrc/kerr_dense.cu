// kerr_dense.cu -- root finding on stored solutions (Sec. 2.2, method (ii)
// of matching a target time): a geodesic integrated in the affine parameter
// with its accepted states stored (kerr_trace_rays_dense) is searched for the
// first stored step across which t passes a target time; on that step the
// state is the cubic Hermite interpolant through both ends and their
// derivatives (dx/dlambda = k, dk/dlambda = the right-hand side of eqs.
// opt0/opti), and the target is solved for on the interpolant by a
// bracketed Newton iteration.
#include "kerr_trace.cuh"
#include "kerr_variants.h"
#include "kerr.h"

#include <algorithm>

namespace {

using namespace kerr;

__device__ __forceinline__ void deriv(double a, const double y[8], double f[8])
{
    f[0] = y[4];
    f[1] = y[5];
    f[2] = y[6];
    f[3] = y[7];
    accel<double>(a, a * a, y[1], y[2], y[3], y[4], y[5], y[6], y[7], f[4], f[5], f[6], f[7]);
}

// Hermite interpolant p(s) on s in [0, 1] of one component and its
// derivative dp/ds: values v0, v1, derivatives d0, d1 (per unit s).
__device__ __forceinline__ void hermite(double s, double v0, double d0, double v1, double d1,
                                        double &p, double &dp)
{
    const double s2 = s * s, s3 = s2 * s;
    p = (2 * s3 - 3 * s2 + 1) * v0 + (s3 - 2 * s2 + s) * d0 + (-2 * s3 + 3 * s2) * v1 +
        (s3 - s2) * d1;
    dp = (6 * s2 - 6 * s) * v0 + (3 * s2 - 4 * s + 1) * d0 + (-6 * s2 + 6 * s) * v1 +
         (3 * s2 - 2 * s) * d1;
}

__global__ void dense_time_kernel(double a, const double *__restrict__ traj, int cap,
                                  const int32_t *__restrict__ count, int64_t n,
                                  const double *__restrict__ t_target, double *__restrict__ y_out,
                                  double *__restrict__ lam_out, int32_t *__restrict__ found)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int m = min((int)count[i], cap);
        const double ts = t_target[i];
        const double *T = traj + (size_t)i * cap * 9;
        int j = -1;
        for (int q = 0; q + 1 < m; ++q) {
            const double d0 = T[q * 9 + 1] - ts, d1 = T[(q + 1) * 9 + 1] - ts;
            if ((d0 <= 0.0 && d1 >= 0.0) || (d0 >= 0.0 && d1 <= 0.0)) {
                j = q;
                break;
            }
        }
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        if (j < 0) {
            for (int c = 0; c < 8; ++c)
                y_out[c * n + i] = nan;
            lam_out[i] = nan;
            found[i] = 0;
            continue;
        }
        const double *A = T + j * 9, *B = T + (j + 1) * 9;
        const double h = B[0] - A[0];
        double f0[8], f1[8];
        deriv(a, A + 1, f0);
        deriv(a, B + 1, f1);
        // solve p_t(s) = ts on [0, 1] (p_t - ts changes sign across it)
        double lo = 0.0, hi = 1.0;
        const double tA = A[1] - ts;
        double s = (B[1] == A[1]) ? 0.0 : (ts - A[1]) / (B[1] - A[1]);
        for (int it = 0; it < 60; ++it) {
            double p, dp;
            hermite(s, A[1], h * f0[0], B[1], h * f1[0], p, dp);
            const double g = p - ts;
            if (fabs(g) <= 1e-13 * (1.0 + fabs(ts)))
                break;
            if ((g < 0.0) == (tA < 0.0))
                lo = s;
            else
                hi = s;
            double sn = dp != 0.0 ? s - g / dp : 0.5 * (lo + hi);
            if (!(sn > lo && sn < hi))
                sn = 0.5 * (lo + hi);
            s = sn;
        }
        for (int c = 0; c < 8; ++c) {
            double p, dp;
            hermite(s, A[1 + c], h * f0[c], B[1 + c], h * f1[c], p, dp);
            y_out[c * n + i] = p;
        }
        lam_out[i] = A[0] + s * h;
        found[i] = 1;
    }
}

bool on_dev(const void *p)
{
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
}

} // namespace

extern "C" int kerr_dense_find_time(double a, const double *traj, int32_t cap,
                                    const int32_t *traj_count, int64_t n, const double *t_target,
                                    double *y_out, double *lam_out, int32_t *found, void *stream)
{
    if (n < 0 || cap < 1 || !(std::fabs(a) <= 1.0))
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_dense_find_time: invalid arguments");
    if (n == 0)
        return KERR_OK;
    if (!traj || !traj_count || !t_target || !y_out || !lam_out || !found)
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_dense_find_time: NULL buffer");
    if (!on_dev(traj) || !on_dev(traj_count) || !on_dev(t_target) || !on_dev(y_out) ||
        !on_dev(lam_out) || !on_dev(found))
        return kerr::kerr_set_error(KERR_EINVAL, "kerr_dense_find_time: buffers must be device memory");
    const int64_t blocks = std::min<int64_t>((n + 127) / 128, 4096);
    dense_time_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(
        a, traj, cap, traj_count, n, t_target, y_out, lam_out, found);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return kerr::kerr_set_error(KERR_ECUDA, cudaGetErrorString(e));
    return KERR_OK;
}
