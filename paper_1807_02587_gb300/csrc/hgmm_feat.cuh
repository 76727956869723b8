// Canonical-frame features of a GMM tree for the learned pose proposal.
//
// Frame of a cloud: c = root mean, s = sqrt(trace Sigma_root) (RMS radius),
// V = the root eigenvectors in columns as the build computed them (the axes
// that seeded the level-0 children), third column negated when det V < 0 so
// that V is a rotation.  Features (64 nodes x 10, BF16): level-0 node k goes
// to group k ^ (4 if the third axis was negated), i.e. the octant of its
// initial mean in the frame; inside a group the live children follow in
// order of decreasing weight (ties by index), and a live level-0 node whose
// children all died stands for itself in the group's first slot.  Entry:
// [64 pi_parent pi_child, V^T (mu - c) / s, 16 upper(V^T Sigma V) / s^2];
// empty slots are zero.  Frame record (16 float64): c, s, V row-major,
// flipped, 0, 0.
#pragma once

#include <cuda_bf16.h>

#include "hgmm_internal.cuh"

namespace hgmm {

constexpr int FEAT_NODES = 64;
constexpr int FEAT_PER_NODE = 10;
constexpr int FEAT_PER_CLOUD = FEAT_NODES * FEAT_PER_NODE;
constexpr int FRAME_DOUBLES = 16;

__device__ __forceinline__ void feat_entry(__nv_bfloat16* out, double w, const double* mu,
                                           const double* S, const double* fr) {
    const double s = fr[3];
    const double* V = fr + 4;  // V[i * 3 + a]: component i of axis a
    const double d[3] = {mu[0] - fr[0], mu[1] - fr[1], mu[2] - fr[2]};
    const double Sf[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
    out[0] = __double2bfloat16(64.0 * w);
    for (int a = 0; a < 3; ++a)
        out[1 + a] = __double2bfloat16((V[a] * d[0] + V[3 + a] * d[1] + V[6 + a] * d[2]) / s);
    // (V^T Sigma V)_ab, upper triangle xx xy xz yy yz zz
    double SV[3][3];
    for (int i = 0; i < 3; ++i)
        for (int b = 0; b < 3; ++b)
            SV[i][b] = Sf[i][0] * V[b] + Sf[i][1] * V[3 + b] + Sf[i][2] * V[6 + b];
    const int ua[6] = {0, 0, 0, 1, 1, 2}, ub[6] = {0, 1, 2, 1, 2, 2};
    const double k = 16.0 / (s * s);
    for (int e = 0; e < 6; ++e) {
        const int a = ua[e], b = ub[e];
        out[4 + e] = __double2bfloat16(k * (V[a] * SV[0][b] + V[3 + a] * SV[1][b] + V[6 + a] * SV[2][b]));
    }
}

// Run by one whole warp; fsm = 16 doubles of shared memory.  Writes the 640
// features and, if frame is not NULL, the frame record.
__device__ inline void tree_features_warp(const RootDev* __restrict__ root,
                                          const NodeStat* __restrict__ stat,
                                          __nv_bfloat16* __restrict__ feat, double* __restrict__ frame,
                                          double* fsm) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        double V[9];
        for (int v = 0; v < 9; ++v) V[v] = root->V[v];
        const double det = V[0] * (V[4] * V[8] - V[5] * V[7]) - V[1] * (V[3] * V[8] - V[5] * V[6]) +
                           V[2] * (V[3] * V[7] - V[4] * V[6]);
        const bool flip = det < 0.0;
        if (flip) {
            V[2] = -V[2];
            V[5] = -V[5];
            V[8] = -V[8];
        }
        const double t = fmax(root->lam[0], 0.0) + fmax(root->lam[1], 0.0) + fmax(root->lam[2], 0.0);
        const double s = t > 0.0 ? sqrt(t) : 1.0;
        for (int a = 0; a < 3; ++a) fsm[a] = root->mu[a];
        fsm[3] = s;
        for (int v = 0; v < 9; ++v) fsm[4 + v] = V[v];
        fsm[13] = flip ? 1.0 : 0.0;
        fsm[14] = 0.0;
        fsm[15] = 0.0;
    }
    __syncwarp();
    if (frame && lane < FRAME_DOUBLES) frame[lane] = fsm[lane];
    for (int i = lane; i < FEAT_PER_CLOUD; i += 32) feat[i] = __float2bfloat16(0.f);
    __syncwarp();
    if (lane < 8) {
        const int k = lane;
        const int group = k ^ (fsm[13] != 0.0 ? 4 : 0);
        __nv_bfloat16* out = feat + group * 8 * FEAT_PER_NODE;
        const NodeStat& P = stat[k];
        if (P.live) {
            int idx[8];
            int nl = 0;
            for (int j = 0; j < 8; ++j)
                if (stat[8 + 8 * k + j].live) idx[nl++] = j;
            // insertion sort: decreasing weight, ties by index
            for (int a = 1; a < nl; ++a) {
                const int x = idx[a];
                const double px = stat[8 + 8 * k + x].pi;
                int b = a - 1;
                while (b >= 0 && stat[8 + 8 * k + idx[b]].pi < px) {
                    idx[b + 1] = idx[b];
                    --b;
                }
                idx[b + 1] = x;
            }
            if (nl == 0) {
                feat_entry(out, P.pi, P.mu, P.S, fsm);
            } else {
                for (int r = 0; r < nl; ++r) {
                    const NodeStat& C = stat[8 + 8 * k + idx[r]];
                    feat_entry(out + r * FEAT_PER_NODE, P.pi * C.pi, C.mu, C.S, fsm);
                }
            }
        }
    }
    __syncwarp();
}

}  // namespace hgmm
