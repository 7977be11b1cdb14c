// Staging of a stage's haloed u_{t-1} tile into shared memory (Sec. 3.1 stage
// input; boundary: half-sample symmetric).
//
// TMA path: one thread issues a tiled bulk tensor copy
// (cp.async.bulk.tensor.3d, box UP x UH x 1 of an [N][H][pitch] float32
// tensor map) whose completion is counted on an mbarrier; every thread waits
// on the mbarrier with a bounded poll.  The copy must start at a column that is
// a multiple of 4 floats (16 bytes), so the box begins at xs = floor4(x0 - 2R)
// and the tile's first column lands at buffer column xoff = (x0 - 2R) - xs.
// Elements outside the image are zero-filled by the copy engine; a fix-up pass
// then writes each of them with its mirror u(sym(y), sym(x)), read from the
// staged box (the mirror lies inside it for every tile geometry the kernels
// use) or, failing that, from global memory.  The result is element for
// element what the symmetric gather stages.
//
// Gather path (no tensor map, or a start column the caller's row reads cannot
// use): every thread loads elements through L2 with the symmetric index, xoff
// = 0.  The persistent batched kernel takes this path: its tiles read data that
// other CTAs wrote earlier in the same launch through the generic proxy.
#pragma once
#include <cuda.h>
#include "common.cuh"
#include "tc_ptx.cuh"

namespace tnrd {

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(tc::smem_u32(bar)), "r"(bytes) : "memory");
}

// Box load of the 3-D tensor map at element coordinates (x, y, z) into dst.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(tc::smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
                   "r"(z), "r"(tc::smem_u32(bar))
                 : "memory");
}

// Stages rows [ys, ys + UH) x columns [xl, xl + UW) of u (image j.u_in, z
// coordinate j.img of j.umap) into sU with row pitch UP = staged_pitch(UW).
// XALIGN: the buffer column of xl must be a multiple of it (2 for float2 row
// reads).  Returns that buffer column, or -1 (uniform over the CTA) if the
// copy did not complete within j.wait_limit cycles; then *j.err is set to
// TNRD_ERR_TIMEOUT, the CTA waits the limit once more for its copy still in
// flight, and sU must not be used.  j.tx_extra (a test hook) arms the mbarrier
// for that many bytes more than the copy brings, so that the waits run out.
// Ends with a CTA barrier.
template <int UH, int UW, int NT, int XALIGN>
__device__ __forceinline__ int stage_u_tile(const TileJob& j, float* sU, int ys, int xl)
{
    constexpr int UP = staged_pitch(UW);
    __shared__ uint64_t bar;
    // u_{t-1} is the previous stage's output, and u_t overwrites the buffer that
    // stage read: wait for it to complete (programmatic dependent launch)
    tc::pdl_wait();
    const int H = j.H, W = j.W;
    const int xs = xl & ~3;
    const int xoff = xl - xs;
    if (j.umap != nullptr && xoff % XALIGN == 0 && (tc::smem_u32(sU) & 127u) == 0) {
        if (threadIdx.x == 0) tc::mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&bar, (uint32_t)(UH * UP * sizeof(float)) + (uint32_t)j.tx_extra);
            tma_load_3d(sU, j.umap, xs, ys, j.img, &bar);
        }
        const bool got = __syncthreads_and(tc::mbar_wait(&bar, 0, j.wait_limit));
        if (!got) {
            if (threadIdx.x == 0) atomicExch(j.err, 4 /* TNRD_ERR_TIMEOUT */);
            tc::mbar_wait(&bar, 0, j.wait_limit);   // let a late copy land before the CTA leaves
            __syncthreads();
            return -1;
        }
        if (ys < 0 || ys + UH > H || xs < 0 || xs + UP > W) {
            for (int idx = threadIdx.x; idx < UH * UP; idx += NT) {
                const int i = idx / UP, c = idx - i * UP;
                const int y = ys + i, x = xs + c;
                if ((unsigned)y < (unsigned)H && (unsigned)x < (unsigned)W) continue;
                const int sy = sym_idx(y, H), sx = sym_idx(x, W);
                const int si = sy - ys, sc = sx - xs;
                sU[idx] = ((unsigned)si < (unsigned)UH && (unsigned)sc < (unsigned)UP)
                              ? sU[si * UP + sc]
                              : __ldcg(j.u_in + (size_t)sy * j.pitch + sx);
            }
            __syncthreads();
        }
        return xoff;
    }
    for (int idx = threadIdx.x; idx < UH * UW; idx += NT) {
        const int i = idx / UW, c = idx - i * UW;
        const int yy = sym_idx(ys + i, H), xx = sym_idx(xl + c, W);
        sU[i * UP + c] = __ldcg(j.u_in + (size_t)yy * j.pitch + xx);
    }
    __syncthreads();
    return 0;
}

}  // namespace tnrd
