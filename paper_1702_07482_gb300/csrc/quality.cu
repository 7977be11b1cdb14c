// Quality indexes of despeckled images (Sec. 4): PSNR, MSSIM, edge
// correlation (EC), mean and variance of the ratio image (RI_M, RI_V) and the
// coefficient of variation of the result (C).  Definitions as stated in
// include/tnrd.h (tnrd_quality).
//
// quality_partials: one CTA per 32 x 32 tile of one image.  The tile of the
// reference x and of the result y is staged (interleaved x, y) with the halo
// both indexes need (1 pixel of symmetric border for the Laplacian, 10 pixels
// right/below for the 11 x 11 SSIM windows whose top-left corner is in the
// tile).  SSIM window statistics in FP32, centred: the window means come from
// a separable 11-tap pass (the 2-D Gaussian is the outer product of the
// normalised 1-D one), then each window's variances and covariance are summed
// directly as sum_w w (x - mx)(y - my), whose terms carry no cancellation (the
// E[x^2] - mx^2 form would need FP64, the slow pipe on this GPU).  Every
// per-pixel quantity is FP32 and each thread sums its 4 pixels in FP32; the
// 256 per-thread partials of each sum are added in FP64 in thread order (one
// thread per sum) and written as the tile's partials.
// quality_finish: one CTA per image sums the tiles' partials in a fixed order
// and forms the indexes.
#include "launch.h"

namespace tnrd {

namespace {

constexpr int QT = 32;                  // tile side (outputs)
constexpr int QWIN = 11;                // SSIM window side
constexpr int QS = QT + QWIN;           // staged side: rows/cols y0-1 .. y0+QT+QWIN-2
constexpr int QHR = QT + QWIN - 1;      // rows of the horizontal pass (42)
constexpr int QNT = 256;

__device__ __forceinline__ int qsym(int i, int n)
{
    const int p = 2 * n;
    int m = i % p;
    m = (m < 0) ? m + p : m;
    return (m < n) ? m : (p - 1 - m);
}

struct QualitySmem {
    float2 xy[QS][QS + 1];   // (x, y) from row y0 - 1, column x0 - 1
    float hm[2][QHR][QT];    // horizontal window sums of x and y
    float mean[2][QT][QT];   // window means of x and y
    float red[QSUMS][QNT + 1];   // per-thread partials (padded: conflict-free column reads)
};

__global__ void __launch_bounds__(QNT) quality_partials(const __grid_constant__ QualityArgs a)
{
    extern __shared__ __align__(16) unsigned char qsmem[];
    QualitySmem& S = *reinterpret_cast<QualitySmem*>(qsmem);
    auto& xy = S.xy;
    auto& hm = S.hm;

    const int n = blockIdx.y;
    const int tx = blockIdx.x % a.tiles_x, ty = blockIdx.x / a.tiles_x;
    const int x0 = tx * QT, y0 = ty * QT;
    const int H = a.H, W = a.W;
    const size_t ioff = (size_t)n * a.img_stride;
    const bool have_ref = a.ref != nullptr, have_noisy = a.noisy != nullptr;
    const float* ref = a.ref + (have_ref ? ioff : 0);
    const float* img = a.img + ioff;
    const float* noisy = a.noisy + (have_noisy ? ioff : 0);

    // staged rows/cols start at y0 - 1 / x0 - 1 (symmetric outside the image)
    for (int e = threadIdx.x; e < QS * QS; e += QNT) {
        const int i = e / QS, j = e - i * QS;
        const size_t o = (size_t)qsym(y0 - 1 + i, H) * a.pitch + qsym(x0 - 1 + j, W);
        xy[i][j] = make_float2(have_ref ? ref[o] : 0.0f, img[o]);
    }
    __syncthreads();

    float acc[QSUMS];
#pragma unroll
    for (int s = 0; s < QSUMS; ++s) acc[s] = 0.0f;

    // pointwise sums over the tile's own pixels
    for (int e = threadIdx.x; e < QT * QT; e += QNT) {
        const int i = e / QT, j = e - i * QT;
        const int yy = y0 + i, xx = x0 + j;
        if (yy >= H || xx >= W) continue;
        const float2 c = xy[i + 1][j + 1];
        const float vy = c.y;
        acc[Q_SY] += vy;
        acc[Q_SYY] = fmaf(vy, vy, acc[Q_SYY]);
        if (have_ref) {
            const float vx = c.x;
            const float d = vx - vy;
            acc[Q_SE] = fmaf(d, d, acc[Q_SE]);
            const float2 u = xy[i][j + 1], dn = xy[i + 2][j + 1], l = xy[i + 1][j], r = xy[i + 1][j + 2];
            const float lx = ((u.x + dn.x) + (l.x + r.x)) - 4.0f * vx;
            const float ly = ((u.y + dn.y) + (l.y + r.y)) - 4.0f * vy;
            acc[Q_LA] += lx;
            acc[Q_LB] += ly;
            acc[Q_LAA] = fmaf(lx, lx, acc[Q_LAA]);
            acc[Q_LBB] = fmaf(ly, ly, acc[Q_LBB]);
            acc[Q_LAB] = fmaf(lx, ly, acc[Q_LAB]);
        }
        if (have_noisy) {
            const float r = noisy[(size_t)yy * a.pitch + xx] / vy;
            acc[Q_R] += r;
            acc[Q_RR] = fmaf(r, r, acc[Q_RR]);
        }
    }

    // SSIM windows with top-left corner (y0 + i, x0 + j), inside the image
    if (have_ref && H >= QWIN && W >= QWIN) {
        for (int e = threadIdx.x; e < QHR * QT; e += QNT) {
            const int i = e / QT, j = e - i * QT;
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int b = 0; b < QWIN; ++b) {
                const float2 v = xy[i + 1][j + 1 + b];
                s0 = fmaf(a.g1[b], v.x, s0);
                s1 = fmaf(a.g1[b], v.y, s1);
            }
            hm[0][i][j] = s0;
            hm[1][i][j] = s1;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < QT * QT; e += QNT) {
            const int i = e / QT, j = e - i * QT;
            float mx = 0.0f, my = 0.0f;
#pragma unroll
            for (int b = 0; b < QWIN; ++b) {
                mx = fmaf(a.g1[b], hm[0][i + b][j], mx);
                my = fmaf(a.g1[b], hm[1][i + b][j], my);
            }
            S.mean[0][i][j] = mx;
            S.mean[1][i][j] = my;
        }
        __syncthreads();
        const float c1 = (0.01f * a.peak) * (0.01f * a.peak), c2 = (0.03f * a.peak) * (0.03f * a.peak);
        for (int e = threadIdx.x; e < QT * QT; e += QNT) {
            const int i = e / QT, j = e - i * QT;
            if (y0 + i > H - QWIN || x0 + j > W - QWIN) continue;
            const float mx = S.mean[0][i][j], my = S.mean[1][i][j];
            float vxx = 0.0f, vyy = 0.0f, vxy = 0.0f;
#pragma unroll
            for (int r = 0; r < QWIN; ++r) {
#pragma unroll
                for (int b = 0; b < QWIN; ++b) {
                    const float2 v = xy[i + 1 + r][j + 1 + b];
                    const float dx = v.x - mx, dy = v.y - my;
                    const float wdx = a.g2[r * QWIN + b] * dx;
                    vxx = fmaf(wdx, dx, vxx);
                    vxy = fmaf(wdx, dy, vxy);
                    vyy = fmaf(a.g2[r * QWIN + b] * dy, dy, vyy);
                }
            }
            acc[Q_SSIM] += ((2.0f * mx * my + c1) * (2.0f * vxy + c2)) /
                           ((fmaf(mx, mx, my * my) + c1) * ((vxx + vyy) + c2));
        }
    }

    // fixed-order reduction: thread s adds sum s's 256 partials in thread order (FP64)
#pragma unroll
    for (int s = 0; s < QSUMS; ++s) S.red[s][threadIdx.x] = acc[s];
    __syncthreads();
    if (threadIdx.x < QSUMS) {
        double t = 0.0;
        for (int k = 0; k < QNT; ++k) t += S.red[threadIdx.x][k];
        a.part[((size_t)n * gridDim.x + blockIdx.x) * QSUMS + threadIdx.x] = t;
    }
}

__global__ void __launch_bounds__(QNT) quality_finish(const __grid_constant__ QualityArgs a,
                                                      int nblocks)
{
    __shared__ double red[QNT];
    __shared__ double tot[QSUMS];
    const int n = blockIdx.x;
    for (int s = 0; s < QSUMS; ++s) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += QNT) t += a.part[((size_t)n * nblocks + b) * QSUMS + s];
        red[threadIdx.x] = t;
        for (int w = QNT / 2; w > 0; w >>= 1) {
            __syncthreads();
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        }
        __syncthreads();
        if (threadIdx.x == 0) tot[s] = red[0];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double np = (double)a.H * a.W;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    double* out = a.out + (size_t)n * QOUT;
    if (a.ref) {
        const double mse = tot[Q_SE] / np;
        out[0] = 10.0 * log10(a.peak * (double)a.peak / mse);
        const double nw = (double)(a.H - QWIN + 1) * (a.W - QWIN + 1);
        out[1] = (a.H >= QWIN && a.W >= QWIN) ? tot[Q_SSIM] / nw : nan;
        const double ca = tot[Q_LAA] - tot[Q_LA] * tot[Q_LA] / np;
        const double cb = tot[Q_LBB] - tot[Q_LB] * tot[Q_LB] / np;
        const double cab = tot[Q_LAB] - tot[Q_LA] * tot[Q_LB] / np;
        out[2] = cab / sqrt(ca * cb);
    } else {
        out[0] = out[1] = out[2] = nan;
    }
    if (a.noisy) {
        const double m = tot[Q_R] / np;
        out[3] = m;
        out[4] = tot[Q_RR] / np - m * m;
    } else {
        out[3] = out[4] = nan;
    }
    const double my = tot[Q_SY] / np;
    out[5] = sqrt(fmax(tot[Q_SYY] / np - my * my, 0.0)) / my;
}

}  // namespace

int quality_tiles(int H, int W) { return ((H + QT - 1) / QT) * ((W + QT - 1) / QT); }

cudaError_t launch_quality(const QualityArgs& a, int N, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(quality_partials, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(QualitySmem));
    if (e != cudaSuccess) return e;
    const int nb = a.tiles_x * a.tiles_y;
    quality_partials<<<dim3(nb, N), QNT, sizeof(QualitySmem), s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    quality_finish<<<N, QNT, 0, s>>>(a, nb);
    return cudaGetLastError();
}

}  // namespace tnrd
