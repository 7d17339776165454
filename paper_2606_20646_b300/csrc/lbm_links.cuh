// Boundary sources and cut-link reconstruction of the FP32 forms (FP32 arithmetic, populations in
// FP32 or BF16), in two kernels (Secs. 3.2-3.4).
//
// k_link_sums: groups of G lanes split each Neumann link's least-squares stencil (the tangent images,
// Eqs. tangent-derivative-2d, tangent-image-3d-lsq), so its index and displacement loads are in flight
// together, and combine the partial sums by shuffles; it holds few registers, so many groups are
// resident.  k_links_f32: one thread per link runs the traction inversion (Eqs. neumann-newton-2d/3d)
// and the reconstruction (Eqs. bfl-eta-ge-half, bfl-eta-lt-half).
//
// Precision.  Near F = I the deformation gradient of a boundary point is I plus a small part, and the
// Neumann rows need F_b - I (the populations are stored shifted by f^eq(0, I)).  Forming F_b in FP32
// and subtracting I would keep only its absolute precision, so everything is carried as small parts:
//   h  = N + hh,  g_a = t_a + gg_a,
//   F_b - I = E + hh (x) N + sum_a gg_a (x) t_a,   E = N (x) N + sum_a t_a (x) t_a - I,
// where E, the defect of the FP32-rounded orthonormal frame, is summed from exact products.  The
// stencil sums gg_a = sum_j w_aj (u_j - u_m) are compensated (exact product and sum errors carried),
// and the stress comes from piola_g, which never forms the terms that cancel near F = I.  The Newton
// state of an FP32 link is hh = h - N.
#pragma once

#include "lbm_kernels.cuh"

namespace tlv {

// boundary value of one boundary condition at t^n + dt/2 (Dirichlet velocity or Neumann traction),
// linear in the link's geometric vector g_l: value = M g_l + k
struct BCTimeF {
    float M[9];
    float k[3];
    int kind;  // 0 Dirichlet, 1 Neumann
    int pad[3];
};
struct BCTimes {
    BCTimeF bc[kMaxBCs];
};

// error-free transformations (round-to-nearest intrinsics keep the compiler from contracting them)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// E = N (x) N + sum_a t_a (x) t_a - I from exact products
template <int D>
__device__ __forceinline__ void frame_defect(const float N[D], const float t[D - 1][D], float E[D * D]) {
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int B = 0; B < D; ++B) {
            float s, err, p, pe, e2;
            two_prod(N[i], N[B], s, err);
            #pragma unroll
            for (int al = 0; al < D - 1; ++al) {
                two_prod(t[al][i], t[al][B], p, pe);
                float ns;
                two_sum(s, p, ns, e2);
                s = ns;
                err = __fadd_rn(err, __fadd_rn(pe, e2));
            }
            E[i * D + B] = __fadd_rn(__fsub_rn(s, i == B ? 1.0f : 0.0f), err);
        }
}

// G_b = F_b - I for the normal-image offset hh
template <int D>
__device__ __forceinline__ void boundary_G(const float E[D * D], const float hh[D], const float N[D],
                                           const float gg[D - 1][D], const float t[D - 1][D], float Gb[D * D]) {
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int B = 0; B < D; ++B) {
            float v = E[i * D + B] + hh[i] * N[B];
            #pragma unroll
            for (int al = 0; al < D - 1; ++al) v += gg[al][i] * t[al][B];
            Gb[i * D + B] = v;
        }
}

// traction residual R = P(I + G_b) N - T and its Jacobian, the acoustic tensor
// Q(N; F_b) = mu I + (lam (J^2 + 1)/2 + mu) a a^T with a = F_b^{-T} N (Eq. acoustic-tensor-general-d);
// false when J <= 0
template <int D>
__device__ __forceinline__ bool traction_rq(const float E[D * D], const float hh[D], const float N[D],
                                            const float gg[D - 1][D], const float t[D - 1][D], const float T[D],
                                            float mu, float lam, float R[D], float Q[D * D]) {
    float Gb[D * D], P[D * D], Fit[D * D];
    boundary_G<D>(E, hh, N, gg, t, Gb);
    const float J = piola_g<float, D>(Gb, mu, lam, P, Fit);
    if (!(J > 0.0f)) return false;
    float av[D];
    #pragma unroll
    for (int i = 0; i < D; ++i) {
        float pn = 0.0f, an = 0.0f;
        #pragma unroll
        for (int A = 0; A < D; ++A) {
            pn += P[i * D + A] * N[A];
            an += Fit[i * D + A] * N[A];
        }
        R[i] = pn - T[i];
        av[i] = an;
    }
    const float kap = 0.5f * lam * (J * J + 1.0f) + mu;
    #pragma unroll
    for (int i = 0; i < D; ++i)
        #pragma unroll
        for (int j = 0; j < D; ++j) Q[i * D + j] = kap * av[i] * av[j] + (i == j ? mu : 0.0f);
    return true;
}

template <int D> constexpr int kLinkLanes = 4;  // lanes per cut link in the stencil sums (8 and 16 measured slower)

// Stencil sums of the Neumann links: one group of G lanes per link splits its LSQ stencil (entries
// r, r + G, ... for lane r), the compensated partial sums are combined by shuffles and lane 0 of the
// group writes gg_a = sum_j w_aj (u_j - u_m) (D - 1 vectors, 8 floats per link).  Few registers, so
// many links' index and displacement loads are in flight on every SM.
template <int D, int G = kLinkLanes<D>>
__global__ void __launch_bounds__(256) k_link_sums(const CutArgs<float> a, float *__restrict__ gsum) {
    const int lane = threadIdx.x & 31, r = lane & (G - 1);
    const unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const long long l = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
    if (l >= a.L.ncut) return;  // whole groups leave together
    const int ns = __ldg(a.L.ns + l);  // 0 for Dirichlet links
    if (ns == 0) return;
    float gh[D - 1][D], ge[D - 1][D];
    #pragma unroll
    for (int al = 0; al < D - 1; ++al)
        #pragma unroll
        for (int i = 0; i < D; ++i) { gh[al][i] = 0.0f; ge[al][i] = 0.0f; }
    float um[D], uml[D];
    un_load<float, D>(a.un, __ldg(a.L.node + l), um, uml);
    constexpr int U = 4;
    const int *__restrict__ sidx = a.L.sidx + l * kLsqCap;
    const float *__restrict__ wl = a.L.w + l * kLsqCap * (D - 1);
    for (int j0 = r; j0 < ns; j0 += U * G) {
        int kk[U];
        float w[U][D - 1], uu[U][D], uul[U][D];
        #pragma unroll
        for (int jj = 0; jj < U; ++jj) {
            const int j = j0 + jj * G < ns ? j0 + jj * G : j0;
            kk[jj] = __ldg(sidx + j);
            TLV_BOUND(kk[jj], a.npad, a.status);
            if constexpr (D == 3) {
                const float2 wv = __ldg(reinterpret_cast<const float2 *>(wl) + j);
                w[jj][0] = wv.x;
                w[jj][1] = wv.y;
            } else {
                w[jj][0] = __ldg(wl + j);
            }
        }
        #pragma unroll
        for (int jj = 0; jj < U; ++jj) un_load<float, D>(a.un, kk[jj], uu[jj], uul[jj]);
        #pragma unroll
        for (int jj = 0; jj < U; ++jj) {
            if (j0 + jj * G >= ns) break;
            #pragma unroll
            for (int i = 0; i < D; ++i) {
                const float du = __fadd_rn(__fsub_rn(uu[jj][i], um[i]), __fsub_rn(uul[jj][i], uml[i]));
                #pragma unroll
                for (int al = 0; al < D - 1; ++al) {
                    float pr, pe, sn, se;
                    two_prod(w[jj][al], du, pr, pe);
                    two_sum(gh[al][i], pr, sn, se);
                    gh[al][i] = sn;
                    ge[al][i] = __fadd_rn(ge[al][i], __fadd_rn(pe, se));
                }
            }
        }
    }
    #pragma unroll
    for (int o = G / 2; o > 0; o >>= 1)
        #pragma unroll
        for (int al = 0; al < D - 1; ++al)
            #pragma unroll
            for (int i = 0; i < D; ++i) {
                const float xh = __shfl_xor_sync(gm, gh[al][i], o), xe = __shfl_xor_sync(gm, ge[al][i], o);
                float sn, se;
                two_sum(gh[al][i], xh, sn, se);
                gh[al][i] = sn;
                ge[al][i] = __fadd_rn(__fadd_rn(ge[al][i], xe), se);
            }
    if (r == 0) {
        float out[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        #pragma unroll
        for (int al = 0; al < D - 1; ++al)
            #pragma unroll
            for (int i = 0; i < D; ++i) out[al * D + i] = __fadd_rn(gh[al][i], ge[al][i]);
        float4 *o4 = reinterpret_cast<float4 *>(gsum + l * 8);
        o4[0] = make_float4(out[0], out[1], out[2], out[3]);
        o4[1] = make_float4(out[4], out[5], out[6], out[7]);
    }
}

// Coefficient of the upstream term of each FP32 link (LinkGeom::cu): D_b,v (1 - 2 eta) for eta < 1/2
// with an active upstream node m - e_c, else 0; D_b,v = +1 for Neumann, -1 for Dirichlet links.
template <int D>
__global__ void k_link_cu(LinkGeom<float> L, const uint8_t *__restrict__ flags, const BCD *__restrict__ bcs) {
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= L.ncut) return;
    const int q = L.q[l];
    const float eta = (float)L.eta[l];
    const bool up = !((flags[L.node[l]] >> (q ^ 1)) & 1);
    const float dv = bcs[L.bc[l]].kind != 0 ? 1.0f : -1.0f;  // kind 1: Neumann
    L.cu[l] = (up && !(eta >= 0.5f)) ? dv * (1.0f - 2.0f * eta) : 0.0f;
}

// One thread per cut link: boundary values, the traction inversion of a Neumann link (its tangent
// images from k_link_sums), and the reconstruction of the K incoming components.
template <int D, typename pop>
__global__ void __launch_bounds__(256) k_links_f32(const CutArgs<float> a, const __grid_constant__ BCTimes bt,
                                                   const float *__restrict__ gsum) {
    constexpr int K = D + D * D;
    const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (l >= a.L.ncut) return;
    const int q = __ldg(a.L.q + l), A = q >> 1;
    const float s = (q & 1) ? -1.0f : 1.0f;  // e = s e_A, d = -e
    const BCTimeF &tb = bt.bc[__ldg(a.L.bc + l)];
    const int mnode = __ldg(a.L.node + l);
    const float eta = (float)__ldg(a.L.eta + l);
    // operands of the reconstruction, loaded first: the node's kept pair f*_c(m), f*_{c^1}(m).  The
    // upstream node's f*_c, which an eta < 1/2 link with an active upstream node m - e_c needs, is the
    // value the next gather pulls for direction c at m: that gather adds its term (cu != 0)
    const float cu = __ldg(a.L.cu + l);
    float fo[K], fi[K];
    vload<K>(a.L.fo + l * (2 * K), fo);
    vload<K>(a.L.fo + l * (2 * K) + K, fi);
    const float4 gv = __ldg(a.L.bvec + l);
    const float gl[3] = {gv.x, gv.y, gv.z};
    float val[D];  // Dirichlet velocity or Neumann traction at X_b, t^n + dt/2
    #pragma unroll
    for (int i = 0; i < D; ++i) val[i] = tb.k[i] + tb.M[3 * i] * gl[0] + tb.M[3 * i + 1] * gl[1] + tb.M[3 * i + 2] * gl[2];
    const float c = (float)a.c;
    float S[K];
    if (tb.kind == 0) {
        // velocity Dirichlet rows (Eqs. dirichlet-rows-curved, dirichlet-compact-curved)
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            S[i] = val[i] * (1.0f / float(D));
            #pragma unroll
            for (int B = 0; B < D; ++B) S[D + i * D + B] = (B == A) ? s * val[i] / c : 0.0f;
        }
    } else {
        // nominal-traction Neumann rows (Eqs. neumann-rows-curved, neumann-compact-curved)
        float mu = a.mtab ? a.mtab[2 * a.mat[mnode]] : (float)a.mu;
        const float lam = a.mtab ? a.mtab[2 * a.mat[mnode] + 1] : (float)a.lam;
        if (a.mu_field) mu = a.mu_field[mnode];
        float N[D], t[D - 1][D], gg[D - 1][D];
        #pragma unroll
        for (int i = 0; i < D; ++i) N[i] = (float)__ldg(a.L.Nb + 3 * l + i);
        #pragma unroll
        for (int al = 0; al < D - 1; ++al)
            #pragma unroll
            for (int i = 0; i < D; ++i) {
                t[al][i] = (float)__ldg(a.L.tan + 6 * l + 3 * al + i);
                gg[al][i] = __ldg(gsum + l * 8 + al * D + i);
            }
        float E[D * D];
        frame_defect<D>(N, t, E);
        float tinf = 0.0f;
        #pragma unroll
        for (int i = 0; i < D; ++i) tinf = fmaxf(tinf, fabsf(val[i]));
        // Newton on hh with the analytic Jacobian, from the previous step's image.  Until |R| <=
        // 2e-6 (mu + lambda + |T|) a halving line search (rejecting det F_b <= 0) secures decrease;
        // then at most two full steps refine while |R| still falls (quadratic convergence reaches the
        // FP32 rounding level of P N - T), and a step that does not lower |R| ends the iteration.
        // |R| above 2e-6 (mu + lambda + |T|) at the end is a failed inversion.
        const float scale = mu + lam + tinf;
        float hh[D], R[D], Jq[D * D];
        #pragma unroll
        for (int i = 0; i < D; ++i) hh[i] = a.L.h[3 * l + i];
        bool ok = traction_rq<D>(E, hh, N, gg, t, val, mu, lam, R, Jq);
        if (!ok) {
            #pragma unroll
            for (int i = 0; i < D; ++i) hh[i] = 0.0f;
            ok = traction_rq<D>(E, hh, N, gg, t, val, mu, lam, R, Jq);
        }
        int refine = 0;
        #pragma unroll 1
        for (int it = 0; ok && it < 16; ++it) {
            float rinf = 0.0f, r2 = 0.0f;
            #pragma unroll
            for (int i = 0; i < D; ++i) { rinf = fmaxf(rinf, fabsf(R[i])); r2 += R[i] * R[i]; }
            if (!isfinite(r2)) { ok = false; break; }
            if (r2 == 0.0f) break;
            const bool near = rinf <= 2e-6f * scale;
            if (near && refine++ == 2) break;
            float mR[D], dh[D];
            #pragma unroll
            for (int i = 0; i < D; ++i) mR[i] = -R[i];
            if (!solve_small<float, D>(Jq, mR, dh)) break;
            float al = 1.0f;
            bool acc = false;
            float ht[D], Rt[D], Jt[D * D];
            const int tries = near ? 1 : 20;  // refinement: the full step only
            #pragma unroll 1
            for (int ls = 0; ls < tries; ++ls) {
                #pragma unroll
                for (int i = 0; i < D; ++i) ht[i] = hh[i] + al * dh[i];
                if (traction_rq<D>(E, ht, N, gg, t, val, mu, lam, Rt, Jt)) {
                    float rt2 = 0.0f;
                    #pragma unroll
                    for (int i = 0; i < D; ++i) rt2 += Rt[i] * Rt[i];
                    if (rt2 < r2) { acc = true; break; }
                }
                al *= 0.5f;
            }
            if (!acc) break;  // no decrease: the residual is at its rounding level
            #pragma unroll
            for (int i = 0; i < D; ++i) { hh[i] = ht[i]; R[i] = Rt[i]; }
            #pragma unroll
            for (int k = 0; k < D * D; ++k) Jq[k] = Jt[k];
        }
        float rinf = 0.0f;
        #pragma unroll
        for (int i = 0; i < D; ++i) rinf = fmaxf(rinf, fabsf(R[i]));
        if (!(ok && rinf <= 2e-6f * scale)) {
            set_status(a.status, kStNewton);
            #pragma unroll
            for (int i = 0; i < D; ++i) hh[i] = a.L.h[3 * l + i];
        } else {
            #pragma unroll
            for (int i = 0; i < D; ++i) a.L.h[3 * l + i] = hh[i];
        }
        float Gb[D * D], Pb[D * D], Fit[D * D];
        boundary_G<D>(E, hh, N, gg, t, Gb);
        piola_g<float, D>(Gb, mu, lam, Pb, Fit);
        #pragma unroll
        for (int i = 0; i < D; ++i) {
            S[i] = s * Pb[i * D + A] / c;  // -d_A P_iA / c with d = -s e_A
            #pragma unroll
            for (int B = 0; B < D; ++B) S[D + i * D + B] = Gb[i * D + B] * (1.0f / float(D));  // (F_b - I)/D, shifted
        }
    }
    // interpolated pair relation for the incoming population f_{c^1}(m) of the next gather:
    // D_b = diag(-I, I) for Dirichlet, diag(I, -I) for Neumann links
    const bool neu = tb.kind != 0;
    float Rk[K];
    #pragma unroll
    for (int k = 0; k < K; ++k) {
        const float Dk = ((k < D) == neu) ? 1.0f : -1.0f;
        if (eta >= 0.5f)
            Rk[k] = (Dk * fo[k] + S[k]) / (2.0f * eta) + (1.0f - 1.0f / (2.0f * eta)) * fi[k];
        else if (cu != 0.0f)
            Rk[k] = Dk * (2.0f * eta * fo[k]) + S[k];  // + D_k (1 - 2 eta) f*_c(m - e_c) in the gather
        else  // no upstream node: f*_c(m) stands in for it
            Rk[k] = Dk * (2.0f * eta * fo[k] + (1.0f - 2.0f * eta) * fo[k]) + S[k];
    }
    vstore<K>(a.L.rec + l * K, Rk);
}

}  // namespace tlv
