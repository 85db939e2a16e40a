// gpv_init.cuh -- covariance-centred initialisation of 3D Gaussians (GS-LIVM
// Sec. 3.2): per n_r x n_r subgrid of a voxel's query nodes, the inverse-variance
// weighted position (Eq. 6) and covariance Phi (Eq. 7), then scale and rotation of the
// Gaussian from Phi = R S S^T R^T (Eq. 5).
//
// Precision: the sums of Eq. 6-7 run in the working type T of the solve (float-float on
// the mixed path), because the smallest eigenvalue of Phi (the surface thickness) can
// sit 1e5 below the largest.  The eigenvectors come from FP32 Jacobi rotations on Phi
// rounded to FP32; each eigenvalue is then the Rayleigh quotient e^T Phi e evaluated in
// T, whose error is quadratic in the eigenvector error.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpv_num.cuh"

namespace gpv {

__device__ __forceinline__ float rs_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rs_sqrt(double x) { return rsqrt(x); }

// Eigen decomposition of a symmetric 3x3 matrix by cyclic two-sided plane rotations
// (Jacobi's method).  a[] holds (00,01,02,11,12,22); on return ev[k] are the
// eigenvalues and columns of E (E[r*3+k]) the eigenvectors.
template <class R>
__device__ inline void sym3_eig(const R a_in[6], R ev[3], R E[9])
{
    R m[3][3] = {{a_in[0], a_in[1], a_in[2]}, {a_in[1], a_in[3], a_in[4]}, {a_in[2], a_in[4], a_in[5]}};
    R V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    // an off-diagonal element below tiny * (|a_pp| + |a_qq|) is set to zero: it moves
    // the eigenvalues by less than its square over the gap and the eigenvectors by less
    // than tiny (|a_pp| + |a_qq|) / gap
    const R tiny = sizeof(R) == 4 ? (R)1e-8 : (R)1e-17;
    for (int it = 0; it < 16; ++it) {
        if (m[0][1] == (R)0 && m[0][2] == (R)0 && m[1][2] == (R)0) break;
#pragma unroll
        for (int pr = 0; pr < 3; ++pr) {
            const int p = pr == 2 ? 1 : 0;
            const int q = pr == 0 ? 1 : 2;
            R apq = m[p][q];
            if (fabs(apq) <= tiny * (fabs(m[p][p]) + fabs(m[q][q]))) {
                m[p][q] = (R)0;
                m[q][p] = (R)0;
                continue;
            }
            // tangent of the rotation angle, smaller root of t^2 + 2 t zeta - 1 = 0
            R zeta = (m[q][q] - m[p][p]) / ((R)2 * apq);
            R t = (R)1 / (fabs(zeta) + sqrt((R)1 + zeta * zeta));
            if (zeta < (R)0) t = -t;
            R c = rs_sqrt((R)1 + t * t);
            R s = t * c;
#pragma unroll
            for (int r = 0; r < 3; ++r) {  // columns p, q of m J
                R x = m[r][p], y = m[r][q];
                m[r][p] = c * x - s * y;
                m[r][q] = s * x + c * y;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {  // rows p, q of J^T (m J)
                R x = m[p][r], y = m[q][r];
                m[p][r] = c * x - s * y;
                m[q][r] = s * x + c * y;
            }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                R x = V[r][p], y = V[r][q];
                V[r][p] = c * x - s * y;
                V[r][q] = s * x + c * y;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ev[k] = m[k][k];
#pragma unroll
        for (int r = 0; r < 3; ++r) E[r * 3 + k] = V[r][k];
    }
}

// Largest-magnitude component made positive (ties: lower index keeps priority).
__device__ inline void orient(float e[3])
{
    int k = 0;
    if (fabsf(e[1]) > fabsf(e[k])) k = 1;
    if (fabsf(e[2]) > fabsf(e[k])) k = 2;
    if (e[k] < 0.f) { e[0] = -e[0]; e[1] = -e[1]; e[2] = -e[2]; }
}

// Unit quaternion (w, x, y, z), w >= 0, of the rotation with columns c0, c1, c2.
__device__ inline void rot_to_quat(const float c0[3], const float c1[3], const float c2[3],
                                   float q[4])
{
    const float r00 = c0[0], r10 = c0[1], r20 = c0[2];
    const float r01 = c1[0], r11 = c1[1], r21 = c1[2];
    const float r02 = c2[0], r12 = c2[1], r22 = c2[2];
    // the largest of 4w^2, 4x^2, 4y^2, 4z^2 gives a stable square root
    const float fw = 1.f + r00 + r11 + r22;
    const float fx = 1.f + r00 - r11 - r22;
    const float fy = 1.f - r00 + r11 - r22;
    const float fz = 1.f - r00 - r11 + r22;
    float w, x, y, z;
    if (fw >= fx && fw >= fy && fw >= fz) {
        w = 0.5f * sqrtf(fw);
        const float f = 0.25f / w;
        x = (r21 - r12) * f; y = (r02 - r20) * f; z = (r10 - r01) * f;
    } else if (fx >= fy && fx >= fz) {
        x = 0.5f * sqrtf(fx);
        const float f = 0.25f / x;
        w = (r21 - r12) * f; y = (r01 + r10) * f; z = (r02 + r20) * f;
    } else if (fy >= fz) {
        y = 0.5f * sqrtf(fy);
        const float f = 0.25f / y;
        w = (r02 - r20) * f; x = (r01 + r10) * f; z = (r12 + r21) * f;
    } else {
        z = 0.5f * sqrtf(fz);
        const float f = 0.25f / z;
        w = (r10 - r01) * f; x = (r02 + r20) * f; y = (r12 + r21) * f;
    }
    float inv = rsqrtf(w * w + x * x + y * y + z * z);
    if (w < 0.f) inv = -inv;
    q[0] = w * inv; q[1] = x * inv; q[2] = y * inv; q[3] = z * inv;
}

// One Gaussian from subgrid (bi, bj) of a voxel.  mv_mean / mv_var hold the voxel's
// G*G predictions in T (query q = i*G + j, value coordinate relative to the voxel
// centre); nodes[] the G grid nodes.  Writes pos (world), scale, quat (w x y z) in FP32.
template <class T>
__device__ inline void init_one_gaussian(const T* mv_mean, const T* mv_var, const T* nodes,
                                         int axis, const float* centre, float size, int G,
                                         int n_s, int n_r, float sf2, int init_mode, int bi,
                                         int bj, float* pos, float* scale, float* quat)
{
    const int p1 = axis == 2 ? 0 : axis + 1;
    const int p2 = axis == 0 ? 2 : (axis == 1 ? 0 : 1);
    const float vfloor = 1e-6f * sf2;
    // Eq. 6: p = sum w P / sum w, weights 1 / max(var, floor) (relative error 2^-24 in
    // the weights changes p and Phi only at that relative level)
    float sw = 0.f;
    T sp[3] = {zero<T>(), zero<T>(), zero<T>()};
    for (int ii = 0; ii < n_r; ++ii) {
        const int i = bi * n_r + ii;
        for (int jj = 0; jj < n_r; ++jj) {
            const int j = bj * n_r + jj;
            const int q = i * G + j;
            const float w = 1.f / fmaxf(to_f(mv_var[q]), vfloor);
            sw += w;
            T P[3];
            P[p1] = nodes[i]; P[p2] = nodes[j]; P[axis] = mv_mean[q];
#pragma unroll
            for (int k = 0; k < 3; ++k) sp[k] = gfma(P[k], from_f<T>(w), sp[k]);
        }
    }
    const T isw = from_f<T>(1.f) / from_f<T>(sw);
    T pc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) pc[k] = sp[k] * isw;
    // Eq. 7: Phi = sum w (P - p)(P - p)^T / sum w
    T c6[6] = {zero<T>(), zero<T>(), zero<T>(), zero<T>(), zero<T>(), zero<T>()};
    for (int ii = 0; ii < n_r; ++ii) {
        const int i = bi * n_r + ii;
        for (int jj = 0; jj < n_r; ++jj) {
            const int j = bj * n_r + jj;
            const int q = i * G + j;
            const float w = 1.f / fmaxf(to_f(mv_var[q]), vfloor);
            T P[3];
            P[p1] = nodes[i]; P[p2] = nodes[j]; P[axis] = mv_mean[q];
            const T d0 = P[0] - pc[0], d1 = P[1] - pc[1], d2 = P[2] - pc[2];
            const T wd0 = d0 * from_f<T>(w), wd1 = d1 * from_f<T>(w), wd2 = d2 * from_f<T>(w);
            c6[0] = gfma(wd0, d0, c6[0]); c6[1] = gfma(wd0, d1, c6[1]);
            c6[2] = gfma(wd0, d2, c6[2]); c6[3] = gfma(wd1, d1, c6[3]);
            c6[4] = gfma(wd1, d2, c6[4]); c6[5] = gfma(wd2, d2, c6[5]);
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) c6[k] = c6[k] * isw;
#pragma unroll
    for (int k = 0; k < 3; ++k) pos[k] = to_f(from_f<T>(centre[k]) + pc[k]);
    if (init_mode == 1) {  // Eq. 8 as printed: diagonal of Phi, identity rotation
        scale[0] = to_f(c6[0]); scale[1] = to_f(c6[3]); scale[2] = to_f(c6[5]);
        quat[0] = 1.f; quat[1] = 0.f; quat[2] = 0.f; quat[3] = 0.f;
        return;
    }
    float f6[6], ev[3], E[9];
#pragma unroll
    for (int k = 0; k < 6; ++k) f6[k] = to_f(c6[k]);
    sym3_eig<float>(f6, ev, E);
    int o0 = 0, o1 = 1, o2 = 2;  // descending order of eigenvalues
    if (ev[o1] > ev[o0]) { int t = o0; o0 = o1; o1 = t; }
    if (ev[o2] > ev[o1]) { int t = o1; o1 = o2; o2 = t; }
    if (ev[o1] > ev[o0]) { int t = o0; o0 = o1; o1 = t; }
    float e1[3] = {E[o0], E[3 + o0], E[6 + o0]};
    float e2[3] = {E[o1], E[3 + o1], E[6 + o1]};
    orient(e1);
    orient(e2);
    float e3[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]};
    // Rayleigh quotients e^T Phi e in T
    const float* cols[3] = {e1, e2, e3};
    const float sfl = 1e-4f * size;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float* e = cols[a];
        const T x = from_f<T>(e[0]), y = from_f<T>(e[1]), z = from_f<T>(e[2]);
        T r = c6[0] * x * x + c6[3] * y * y + c6[5] * z * z;
        r = r + from_f<T>(2.f) * (c6[1] * x * y + c6[2] * x * z + c6[4] * y * z);
        const float nn = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        const float lam = to_f(r) / nn;
        scale[a] = sqrtf(fmaxf(lam, sfl * sfl));
    }
    float q[4];
    rot_to_quat(e1, e2, e3, q);
    quat[0] = q[0]; quat[1] = q[1]; quat[2] = q[2]; quat[3] = q[3];
}

}  // namespace gpv
