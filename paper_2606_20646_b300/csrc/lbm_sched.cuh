// Setup of the overlapped link schedule: the window list split into boundary windows, which hold
// a node the link kernels read or feed, and the others, which share no data with the link kernels
// and run alongside them.
#pragma once

#include "lbm_kernels.cuh"

namespace tlv {

// Window classes for running the link kernels alongside the regular step.  A window is a boundary
// window when a node of it is read or fed by the link kernels: a cut node (its kept pair, its
// reconstructed populations), a node whose u^n a Neumann stencil reads (kNeedU), or the upstream
// node m - e_q of a cut link (m, q) (its post-collision populations, for eta < 1/2).  One warp per
// window; cls[s] = 1 for a boundary window.
static __global__ void k_seg_class(Box b, const int2 *__restrict__ seg, int nseg, const uint8_t *__restrict__ flags,
                                   int *cls) {
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= nseg) return;
    const int lane = threadIdx.x & 31;
    const int2 sg = seg[s];
    const int x = sg.x - sg.y * b.nx + lane;
    bool mark = false;
    if (x < b.nx) {
        const int node = sg.x + lane;
        const uint8_t fl = flags[node];
        if (fl & kActive) {
            mark = (fl & (kCutMask | kNeedU)) != 0;
            const int y = sg.y % b.ny, z = sg.y / b.ny;
            for (int q = 0; q < 2 * b.D && !mark; ++q) {
                if ((fl >> q) & 1) continue;  // no active neighbour that way
                const int nb = nbr(b, node, x, y, z, q);
                mark = (flags[nb] >> q) & 1;  // link (node + e_q, q) is cut: this node is its upstream node
            }
        }
    }
    mark = __any_sync(0xffffffffu, mark);
    if (lane == 0) cls[s] = mark ? 1 : 0;
}

// stable partition of the window list: boundary windows first (pos = exclusive scan of cls), then
// the others, each class in list order
static __global__ void k_seg_partition(const int2 *__restrict__ seg, int nseg, const int *__restrict__ cls,
                                       const int *__restrict__ pos, int2 *out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    const int nb = pos[nseg - 1] + cls[nseg - 1];
    out[cls[s] ? pos[s] : nb + (s - pos[s])] = seg[s];
}

}  // namespace tlv
