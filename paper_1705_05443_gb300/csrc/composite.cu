// composite.cu -- products of Section 6 built from H^2 matvecs of the same
// representation: the Cauchy-like matrix of Section 6.3 and the double-layer
// (Nystrom) matrix of Section 6.4.
//
// A Cauchy-like matrix with generators w (nx x p) and v (ny x p) has the
// entries (6.1) a_ij = kappa(x_i, y_j) sum_l w_il v_jl, i.e. (6.2)
// A = sum_l diag(w_l) C diag(v_l) with C = [kappa(x_i, y_j)].  With the H^2
// representation C^ of C, A X = sum_l diag(w_l) (C^ (diag(v_l) X)): the p
// scaled copies of X are applied as one block of p * nrhs right-hand sides
// and recombined row by row.  (The paper merges the generators of the p
// scaled representations instead; for the product the two are the same.)
#include "internal.cuh"

namespace smash {

// Xp[j, l * nrhs + c] = v[j, l] X[j, c]
__global__ void cl_scale_kernel(const double *__restrict__ X, const double *__restrict__ v, int64_t ny, int p,
                                int nrhs, double *__restrict__ Xp) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t w = (int64_t)p * nrhs;
    if (t >= ny * w) return;
    const int64_t j = t / w;
    const int rem = (int)(t - j * w), l = rem / nrhs, c = rem - l * nrhs;
    Xp[t] = v[j * p + l] * X[j * nrhs + c];
}

// Y[i, c] = sum_l w[i, l] Yp[i, l * nrhs + c], summed in the order of l
__global__ void cl_combine_kernel(const double *__restrict__ Yp, const double *__restrict__ w, int64_t nx, int p,
                                  int nrhs, double *__restrict__ Y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nx * nrhs) return;
    const int64_t i = t / nrhs;
    const int c = (int)(t - i * nrhs);
    const double *yr = Yp + i * (int64_t)p * nrhs;
    double s = 0.0;
    for (int l = 0; l < p; ++l) s += w[i * p + l] * yr[(int64_t)l * nrhs + c];
    Y[t] = s;
}

// Double layer (6.7)/(6.9): the y-gradient kernels applied to the
// components of nu(y_j) w_j.  X1 = diag(nu_1 w) X, X2 = diag(nu_2 w) X.
__global__ void dl_scale_kernel(const double *__restrict__ X, const double *__restrict__ nu,
                                const double *__restrict__ wts, int64_t ny, int nrhs, double *__restrict__ X1,
                                double *__restrict__ X2) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ny * nrhs) return;
    const int64_t j = t / nrhs;
    const double x = X[t], w = wts[j];
    X1[t] = (nu[2 * j] * w) * x;
    X2[t] = (nu[2 * j + 1] * w) * x;
}

// Y = (Y1 + Y2) + diag(dg) X  (dg may be NULL)
__global__ void dl_combine_kernel(const double *__restrict__ Y1, const double *__restrict__ Y2,
                                  const double *__restrict__ dg, const double *__restrict__ X, int64_t n, int nrhs,
                                  double *__restrict__ Y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * nrhs) return;
    double v = Y1[t] + Y2[t];
    if (dg) v += dg[t / nrhs] * X[t];
    Y[t] = v;
}

static bool on_device(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace smash

using namespace smash;

extern "C" {

smash_status smash_matvec_cauchy_like(smash_handle h, const double *w, const double *v, int p, const double *X,
                                      double *Y, int nrhs, int precision, void *stream) {
    try {
        if (!w || !v) fail(SMASH_EINVAL, "generators w or v are NULL");
        if (p < 1) fail(SMASH_EINVAL, "p must be >= 1");
        if (nrhs < 1 || (int64_t)p * nrhs > kMaxNrhs)
            fail(SMASH_EINVAL, "p * nrhs must be in [1, %d]", kMaxNrhs);
        check_matvec_args(h, X, Y, p * nrhs, precision);
        cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
        Arena tmp(s);
        auto to_dev = [&](const double *src, size_t n) -> const double * {
            if (on_device(src)) return src;
            double *d = tmp.alloc<double>(n);
            CK(cudaMemcpyAsync(d, src, n * sizeof(double), cudaMemcpyHostToDevice, s));
            return d;
        };
        const double *wd = to_dev(w, (size_t)h->nx * p);
        const double *vd = to_dev(v, (size_t)h->ny * p);
        const double *Xd = to_dev(X, (size_t)h->ny * nrhs);
        const bool yhost = !on_device(Y);
        double *Yd = yhost ? tmp.alloc<double>((size_t)h->nx * nrhs) : Y;
        double *Xp = tmp.alloc<double>((size_t)h->ny * p * nrhs);
        double *Yp = tmp.alloc<double>((size_t)h->nx * p * nrhs);
        const int64_t n1 = h->ny * (int64_t)p * nrhs, n2 = h->nx * (int64_t)nrhs;
        cl_scale_kernel<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(Xd, vd, h->ny, p, nrhs, Xp);
        LAUNCHED();
        run_matvec(h, Xp, Yp, p * nrhs, precision, s, nullptr);
        cl_combine_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(Yp, wd, h->nx, p, nrhs, Yd);
        LAUNCHED();
        if (yhost) CK(cudaMemcpyAsync(Y, Yd, (size_t)h->nx * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        tmp.release();
        if (yhost || !stream) CK(cudaStreamSynchronize(s));
        return SMASH_OK;
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return SMASH_ENOMEM;
    }
}

smash_status smash_matvec_double_layer(smash_handle h, const double *nu, const double *wts, const double *diag,
                                       const double *X, double *Y, int nrhs, int precision, void *stream) {
    try {
        if (!nu || !wts) fail(SMASH_EINVAL, "normals or weights are NULL");
        check_matvec_args(h, X, Y, nrhs, precision, SMASH_K_DLP1);
        if (h->nx != h->ny) fail(SMASH_EINVAL, "the double-layer matrix needs X = Y (a Nystrom discretisation)");
        cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
        Arena tmp(s);
        auto to_dev = [&](const double *src, size_t n) -> const double * {
            if (!src || on_device(src)) return src;
            double *d = tmp.alloc<double>(n);
            CK(cudaMemcpyAsync(d, src, n * sizeof(double), cudaMemcpyHostToDevice, s));
            return d;
        };
        const int64_t n = h->nx;
        const double *nud = to_dev(nu, (size_t)n * 2);
        const double *wd = to_dev(wts, (size_t)n);
        const double *dgd = to_dev(diag, (size_t)n);
        const double *Xd = to_dev(X, (size_t)n * nrhs);
        const bool yhost = !on_device(Y);
        double *Yd = yhost ? tmp.alloc<double>((size_t)n * nrhs) : Y;
        double *X1 = tmp.alloc<double>((size_t)n * nrhs), *X2 = tmp.alloc<double>((size_t)n * nrhs);
        double *Y1 = tmp.alloc<double>((size_t)n * nrhs), *Y2 = tmp.alloc<double>((size_t)n * nrhs);
        const unsigned blocks = (unsigned)((n * nrhs + 255) / 256);
        dl_scale_kernel<<<blocks, 256, 0, s>>>(Xd, nud, wd, n, nrhs, X1, X2);
        LAUNCHED();
        run_matvec(h, X1, Y1, nrhs, precision, s, nullptr, SMASH_K_DLP1);
        run_matvec(h, X2, Y2, nrhs, precision, s, nullptr, SMASH_K_DLP2);
        dl_combine_kernel<<<blocks, 256, 0, s>>>(Y1, Y2, dgd, Xd, n, nrhs, Yd);
        LAUNCHED();
        if (yhost) CK(cudaMemcpyAsync(Y, Yd, (size_t)n * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
        tmp.release();
        if (yhost || !stream) CK(cudaStreamSynchronize(s));
        return SMASH_OK;
    } catch (const Error &e) {
        set_last_error(e.msg.c_str());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return SMASH_ENOMEM;
    }
}

}  // extern "C"
