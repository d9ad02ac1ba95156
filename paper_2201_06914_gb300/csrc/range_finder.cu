// Range-finder probes on the device (Sec. 2.1): [Q, ~] = qr(A Z) with A = (D D^T)^p, the
// power-iteration form of the randomized range finder, for a batch of shots.
//
// D is an nt x ncols matrix per shot (or one shared by all shots): the shot's data
// (ncols = receivers) or the causal convolution matrix of the source wavelet (ncols = nt),
// the two readings of A this library offers.  The two products of each power step,
// T = D^T Y and Y = D T, run on the tensor-core probe contraction (probe_gemm.cu); this
// file holds what is left: a tiled transpose and a thin QR by classical Gram-Schmidt with
// one full reorthogonalisation (CGS2) in FP64, one CTA per shot.  CGS2 gives Q orthonormal
// to working precision for any numerically full-rank Y and the positive diagonal of R
// (the sign convention of the oracle's qr).  Y is re-orthonormalised after every power
// step; in exact arithmetic that leaves the final Q unchanged (the intermediate R factors
// only multiply the sketch from the right by triangular matrices with positive diagonals).
#include "wp_internal.cuh"

namespace wp {

// out[s][c][r] = in[s][r][c] for an R x C matrix per shot (32 x 32 tiles through shared
// memory, both sides coalesced).
__global__ void transpose_kernel(const float *__restrict__ in, long long in_ss, int R, int C,
                                 float *__restrict__ out, long long out_ss)
{
    __shared__ float tile[32][33];
    const long long s = blockIdx.z;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const float *src = in + s * in_ss;
    float *dst = out + s * out_ss;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[k][threadIdx.x] = src[(long long)r * C + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < R && c < C) dst[(long long)c * R + r] = tile[threadIdx.x][k];
    }
}

cudaError_t launch_transpose(const float *in, long long in_ss, int R, int C, int nmat, float *out,
                             long long out_ss, cudaStream_t s)
{
    dim3 grid((C + 31) / 32, (R + 31) / 32, nmat);
    transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(in, in_ss, R, C, out, out_ss);
    count_launch();
    return cudaGetLastError();
}

constexpr int QR_THREADS = 512;

// Thin QR of Y (nt x r per shot, given column-major as Yt[s][i][t]) by CGS2 in FP64.
// W[s][i][t] is FP64 scratch.  Writes Q[s][t][i] (row-major, the probe layout) and raises
// *err (value 3) when a column has no component left outside the span of the previous
// ones (a rank-deficient sketch); that column is written as zero.
__global__ void __launch_bounds__(QR_THREADS) cgs2_qr_kernel(const float *__restrict__ Yt, int nt, int r,
                                                             double *__restrict__ W, float *__restrict__ Q,
                                                             int *err)
{
    __shared__ double coef[512];
    __shared__ double red[QR_THREADS / 32];
    const long long s = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = QR_THREADS / 32;
    const long long n = (long long)nt * r;
    double *Ws = W + s * n;
    const float *Ys = Yt + s * n;
    for (long long k = tid; k < n; k += QR_THREADS) Ws[k] = (double)Ys[k];
    __syncthreads();
    for (int j = 0; j < r; j++) {
        double *wj = Ws + (long long)j * nt;
        for (int pass = 0; pass < 2; pass++) {
            // coefficients of the previous (orthonormal) columns, one warp per column
            for (int i = warp; i < j; i += nw) {
                const double *qi = Ws + (long long)i * nt;
                double acc = 0.0;
                for (int t = lane; t < nt; t += 32) acc = fma(qi[t], wj[t], acc);
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) coef[i] = acc;
            }
            __syncthreads();
            for (int t = tid; t < nt; t += QR_THREADS) {
                double v = wj[t];
                for (int i = 0; i < j; i++) v = fma(-coef[i], Ws[(long long)i * nt + t], v);
                wj[t] = v;
            }
            __syncthreads();
        }
        double acc = 0.0;
        for (int t = tid; t < nt; t += QR_THREADS) acc = fma(wj[t], wj[t], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (warp == 0) {
            double v = lane < nw ? red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[0] = v;
        }
        __syncthreads();
        const double nrm = sqrt(red[0]);
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        if (tid == 0 && !(nrm > 0.0)) atomicExch(err, 3);
        for (int t = tid; t < nt; t += QR_THREADS) wj[t] *= inv;
        __syncthreads();
    }
    float *Qs = Q + s * n;
    for (long long k = tid; k < n; k += QR_THREADS) {
        const long long t = k / r;
        const int i = (int)(k - t * r);
        Qs[k] = (float)Ws[(long long)i * nt + t];
    }
}

cudaError_t launch_cgs2_qr(const float *Yt, int nt, int r, int nshots, double *W, float *Q, int *err,
                           cudaStream_t s)
{
    if (r > 512) return cudaErrorInvalidValue;
    cgs2_qr_kernel<<<nshots, QR_THREADS, 0, s>>>(Yt, nt, r, W, Q, err);
    count_launch();
    return cudaGetLastError();
}

}  // namespace wp
