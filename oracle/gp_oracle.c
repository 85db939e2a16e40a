/*
 * gp_oracle.c -- plain FP64 CPU oracle for Voxel-GPR and the covariance-centred
 * initialisation of 3D Gaussians (GS-LIVM, arXiv 2410.17084, Sec. 3.1-3.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * product path never links, calls or includes anything from this directory,
 * and this file shares no code, header, table or constant generator with it.
 *
 * Every routine is written for a reader who checks it against the paper:
 * textbook loops, full n x n matrices, no blocking, no fusion, no reordering
 * beyond the definitions cited next to each function.
 *
 * Readings of the paper used here, where it is silent or ambiguous:
 *   - kernel: k(a,b) = sf2 * exp(-lambda * |a-b|^2) (Sec. 3.1; the paper's
 *     setting is lambda = 1, sf2 = 1; a lengthscale l maps to 1/(2 l^2));
 *   - noise: sigma^2 = sn2 on the Gram diagonal (Eq. 2);
 *   - prior mean: mean_mode 1 subtracts the data mean of f and adds it back,
 *     mean_mode 0 is the zero-mean form of Eq. 2;
 *   - the Gram is kappa(x, x) (Alg. 1 prints kappa(x, x*) for K, which
 *     contradicts the definition of K_alpha in Sec. 3.1);
 *   - only the diagonal of Sigma* is produced (Sec. 3.2 uses Sigma*_i alone);
 *   - the "eigenvector" of Sec. 3.1 is the surface normal (smallest
 *     eigenvalue); the value axis is argmax |normal_k|, exact ties prefer
 *     Z, then X, then Y;
 *   - parameter axes follow Alg. 1: X -> (y, z), Y -> (z, x), Z -> (x, y);
 *   - query grid: G = n_s * n_r cell-centred nodes per side of the voxel
 *     face, u_i = -s/2 + (i + 1/2) s / G in voxel-local coordinates;
 *   - weights w = 1 / max(var, 1e-6 sf2) (Eq. 6 with a floor);
 *   - init_mode 0: scale = sqrt(max(eig, (1e-4 s)^2)) with the eigenvectors
 *     of Phi as rotation; init_mode 1: the paper's S = diag(Phi), R = I (Eq. 8).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GPO_OK 0
#define GPO_BELOW_TAU 1
#define GPO_NOT_SPD 4

/* ------------------------------------------------------------------ */
/* 3x3 symmetric eigen decomposition by cyclic Jacobi rotations.      */
/* A is read only.  On return evals[k] is an eigenvalue and column k  */
/* of V (V[r][k]) its unit eigenvector.  Order is not sorted.         */
/* ------------------------------------------------------------------ */
static void jacobi3(const double A_in[3][3], double evals[3], double V[3][3])
{
    double A[3][3];
    memcpy(A, A_in, sizeof(A));
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) V[r][c] = (r == c) ? 1.0 : 0.0;

    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double diag = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation angle that zeroes A[p][q] */
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) /
                           (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                /* A <- J^T A J with J the (p,q) plane rotation */
                for (int k = 0; k < 3; ++k) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int k = 0; k < 3; ++k) evals[k] = A[k][k];
}

/* Exposed for the closed-form pin of the 3x3 eigen solver. */
int gpo_eig3(const double* A9, double* evals, double* V9)
{
    double A[3][3], V[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) A[r][c] = A9[3 * r + c];
    jacobi3(A, evals, V);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) V9[3 * r + c] = V[r][c];
    return GPO_OK;
}

/* ------------------------------------------------------------------ */
/* ALG.HASH of Alg. 2: the voxel index of a point is floor(p / size)  */
/* per coordinate, evaluated in FP32 with IEEE division (the keys are */
/* integers, so both sides must take this decision in the same type). */
/* ------------------------------------------------------------------ */
void gpo_voxel_key(const float* xyz, int64_t npts, float size, int32_t* keys3)
{
    for (int64_t i = 0; i < npts; ++i)
        for (int c = 0; c < 3; ++c) {
            float q = xyz[3 * i + c] / size;
            keys3[3 * i + c] = (int32_t)floorf(q);
        }
}

/* Voxel centre of an integer key, in FP32: ((float)k + 0.5f) * size. */
void gpo_voxel_centre(const int32_t* keys3, int64_t nvox, float size, float* centres)
{
    for (int64_t i = 0; i < 3 * nvox; ++i)
        centres[i] = ((float)keys3[i] + 0.5f) * size;
}

/* ------------------------------------------------------------------ */
/* ALG.PCA and the value-axis switch (Sec. 3.1, Alg. 1 switch).       */
/* normal = eigenvector of the smallest eigenvalue of the points'     */
/* covariance; value axis = the coordinate axis with the smallest     */
/* angle to it = argmax |normal_k|; exact ties prefer Z, then X, Y.   */
/* Returns the axis; also reports the normal and sorted eigenvalues.  */
/* ------------------------------------------------------------------ */
int gpo_pca_axis(const float* xyz, int64_t n, double* normal_out, double* evals_out)
{
    double c[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) c[k] += (double)xyz[3 * i + k];
    for (int k = 0; k < 3; ++k) c[k] /= (double)n;

    double C[3][3] = {{0}};
    for (int64_t i = 0; i < n; ++i) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = (double)xyz[3 * i + k] - c[k];
        for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) C[r][s] += d[r] * d[s];
    }
    for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) C[r][s] /= (double)n;

    double ev[3], V[3][3];
    jacobi3(C, ev, V);
    int kmin = 0;
    for (int k = 1; k < 3; ++k)
        if (ev[k] < ev[kmin]) kmin = k;
    double nrm[3] = {V[0][kmin], V[1][kmin], V[2][kmin]};

    /* preference order Z, X, Y: a later axis wins only if strictly larger */
    const int order[3] = {2, 0, 1};
    int axis = order[0];
    for (int t = 1; t < 3; ++t)
        if (fabs(nrm[order[t]]) > fabs(nrm[axis])) axis = order[t];

    if (normal_out)
        for (int k = 0; k < 3; ++k) normal_out[k] = nrm[k];
    if (evals_out) {
        double s[3] = {ev[0], ev[1], ev[2]};
        for (int a = 0; a < 3; ++a) /* sort ascending */
            for (int b = a + 1; b < 3; ++b)
                if (s[b] < s[a]) { double t = s[a]; s[a] = s[b]; s[b] = t; }
        for (int k = 0; k < 3; ++k) evals_out[k] = s[k];
    }
    return axis;
}

/* Parameter axes of Alg. 1: X -> (y, z), Y -> (z, x), Z -> (x, y). */
static void param_axes(int axis, int* p1, int* p2)
{
    *p1 = (axis + 1) % 3;
    *p2 = (axis + 2) % 3;
}

/* Cell-centred query node i of G over a face of side s (voxel-local). */
static double grid_node(int i, int G, double s)
{
    return -0.5 * s + ((double)i + 0.5) * s / (double)G;
}

/* Textbook unblocked Cholesky A = L L^T of a full n x n row-major SPD     */
/* matrix, in place (lower triangle).  Returns 0, or -1 at a non-positive  */
/* pivot.                                                                  */
static int cholesky(double* A, int64_t n)
{
    for (int64_t j = 0; j < n; ++j) {
        double d = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
        if (!(d > 0.0)) return -1;
        double ljj = sqrt(d);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double s = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* Forward substitution L y = b (L lower, row-major full storage). */
static void forward_sub(const double* L, int64_t n, const double* b, double* y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
}

/* Back substitution L^T x = y. */
static void backward_sub(const double* L, int64_t n, const double* y, double* x)
{
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
}

/* ------------------------------------------------------------------ */
/* Voxel-GPR of one voxel (Alg. 1 body, Sec. 3.1 Eq. 2-3).           */
/*                                                                    */
/* xyz: n world points (FP32, row-major [n,3]); centre: voxel centre; */
/* size: voxel side s; G: query nodes per side; lambda, sf2, sn2:     */
/* kernel and noise; mean_mode as in the header; axis_override in     */
/* {0,1,2} replaces the PCA decision (used only for axis-ambiguous    */
/* voxels), -1 keeps it.                                              */
/* Outputs: *axis_out, mean[G*G] (value coordinate in the voxel-local */
/* frame) and var[G*G] = diag(Sigma*), query q = i*G + j, i on the    */
/* first parameter axis, j on the second.                             */
/* Returns GPO_OK or GPO_NOT_SPD.                                     */
/* ------------------------------------------------------------------ */
int gpo_solve_voxel(const float* xyz, int64_t n, const float* centre, double size, int G,
                    double lambda, double sf2, double sn2, int mean_mode, int axis_override,
                    int* axis_out, double* mean, double* var)
{
    int axis = axis_override >= 0 ? axis_override : gpo_pca_axis(xyz, n, NULL, NULL);
    int p1, p2;
    param_axes(axis, &p1, &p2);
    *axis_out = axis;

    double* x1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* x2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* fm = (double*)malloc(sizeof(double) * (size_t)n);
    double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* alpha = (double*)malloc(sizeof(double) * (size_t)n);
    double* k = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);

    /* voxel-local training inputs x (parameter axes) and targets f (value axis) */
    for (int64_t i = 0; i < n; ++i) {
        x1[i] = (double)xyz[3 * i + p1] - (double)centre[p1];
        x2[i] = (double)xyz[3 * i + p2] - (double)centre[p2];
        fm[i] = (double)xyz[3 * i + axis] - (double)centre[axis];
    }
    double m = 0.0;
    if (mean_mode == 1) {
        for (int64_t i = 0; i < n; ++i) m += fm[i];
        m /= (double)n;
    }
    for (int64_t i = 0; i < n; ++i) fm[i] -= m;

    /* K + sigma^2 I of Eq. 2 */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double d1 = x1[i] - x1[j], d2 = x2[i] - x2[j];
            A[i * n + j] = sf2 * exp(-lambda * (d1 * d1 + d2 * d2)) + (i == j ? sn2 : 0.0);
        }

    int status = GPO_OK;
    if (cholesky(A, n) != 0) {
        status = GPO_NOT_SPD;
        for (int q = 0; q < G * G; ++q) { mean[q] = NAN; var[q] = NAN; }
        goto done;
    }
    /* alpha = (K + sigma^2 I)^-1 (f - m) */
    forward_sub(A, n, fm, y);
    backward_sub(A, n, y, alpha);

    /* Eq. 3 at every query node: mu = m + k^T alpha, var = sf2 - |L^-1 k|^2 */
    for (int i = 0; i < G; ++i) {
        double u = grid_node(i, G, size);
        for (int j = 0; j < G; ++j) {
            double v = grid_node(j, G, size);
            double mu = m;
            for (int64_t t = 0; t < n; ++t) {
                double d1 = x1[t] - u, d2 = x2[t] - v;
                k[t] = sf2 * exp(-lambda * (d1 * d1 + d2 * d2));
                mu += k[t] * alpha[t];
            }
            forward_sub(A, n, k, z);
            double zz = 0.0;
            for (int64_t t = 0; t < n; ++t) zz += z[t] * z[t];
            double vv = sf2 - zz;
            mean[i * G + j] = mu;
            var[i * G + j] = vv > 0.0 ? vv : 0.0;
        }
    }
done:
    free(x1); free(x2); free(fm); free(A); free(y); free(alpha); free(k); free(z);
    return status;
}

/* ------------------------------------------------------------------ */
/* Voxel-GPR with a noise variance per training point (Sec. 3.3: the   */
/* points of an active voxel carry the variance estimated by its last  */
/* solve, new points the sensor variance): A = K + diag(noise).        */
/* Besides mean/var at the query nodes (as gpo_solve_voxel) it returns  */
/* pvar[i], the posterior variance at training input x_i from its      */
/* definition sf2 - k_i^T A^-1 k_i with k_i = (k(x_i, x_j))_j (no noise),  */
/* computed as sf2 - |L^-1 k_i|^2.                                     */
/* ------------------------------------------------------------------ */
int gpo_solve_voxel_hetero(const float* xyz, int64_t n, const float* centre, double size, int G,
                           double lambda, double sf2, const double* noise, int mean_mode,
                           int axis_override, int* axis_out, double* mean, double* var,
                           double* pvar)
{
    int axis = axis_override >= 0 ? axis_override : gpo_pca_axis(xyz, n, NULL, NULL);
    int p1, p2;
    param_axes(axis, &p1, &p2);
    *axis_out = axis;

    double* x1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* x2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* fm = (double*)malloc(sizeof(double) * (size_t)n);
    double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* alpha = (double*)malloc(sizeof(double) * (size_t)n);
    double* k = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);

    for (int64_t i = 0; i < n; ++i) {
        x1[i] = (double)xyz[3 * i + p1] - (double)centre[p1];
        x2[i] = (double)xyz[3 * i + p2] - (double)centre[p2];
        fm[i] = (double)xyz[3 * i + axis] - (double)centre[axis];
    }
    double m = 0.0;
    if (mean_mode == 1) {
        for (int64_t i = 0; i < n; ++i) m += fm[i];
        m /= (double)n;
    }
    for (int64_t i = 0; i < n; ++i) fm[i] -= m;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double d1 = x1[i] - x1[j], d2 = x2[i] - x2[j];
            A[i * n + j] = sf2 * exp(-lambda * (d1 * d1 + d2 * d2)) + (i == j ? noise[i] : 0.0);
        }
    int status = GPO_OK;
    if (cholesky(A, n) != 0) {
        status = GPO_NOT_SPD;
        goto done;
    }
    forward_sub(A, n, fm, y);
    backward_sub(A, n, y, alpha);
    for (int i = 0; i < G; ++i) {
        double u = grid_node(i, G, size);
        for (int j = 0; j < G; ++j) {
            double v = grid_node(j, G, size);
            double mu = m;
            for (int64_t t = 0; t < n; ++t) {
                double d1 = x1[t] - u, d2 = x2[t] - v;
                k[t] = sf2 * exp(-lambda * (d1 * d1 + d2 * d2));
                mu += k[t] * alpha[t];
            }
            forward_sub(A, n, k, z);
            double zz = 0.0;
            for (int64_t t = 0; t < n; ++t) zz += z[t] * z[t];
            double vv = sf2 - zz;
            mean[i * G + j] = mu;
            var[i * G + j] = vv > 0.0 ? vv : 0.0;
        }
    }
    for (int64_t i = 0; i < n; ++i) {  /* posterior variance at the training inputs */
        for (int64_t t = 0; t < n; ++t) {
            double d1 = x1[t] - x1[i], d2 = x2[t] - x2[i];
            k[t] = sf2 * exp(-lambda * (d1 * d1 + d2 * d2));
        }
        forward_sub(A, n, k, z);
        double zz = 0.0;
        for (int64_t t = 0; t < n; ++t) zz += z[t] * z[t];
        double vv = sf2 - zz;
        pvar[i] = vv > 0.0 ? vv : 0.0;
    }
done:
    free(x1); free(x2); free(fm); free(A); free(y); free(alpha); free(k); free(z);
    return status;
}

/* ------------------------------------------------------------------ */
/* Full posterior covariance of the query nodes (Eq. 3, Sigma* of the  */
/* supplementary Alg. 3): cov[q][q'] = k(x*_q, x*_q') - k_q^T A^-1 k_q' */
/* with A = K + sn2 I, evaluated from its definition through z_q =     */
/* L^-1 k_q: cov[q][q'] = k(x*_q, x*_q') - z_q . z_q'.  mean as in     */
/* gpo_solve_voxel.  cov is G^2 x G^2 row-major.                       */
/* ------------------------------------------------------------------ */
int gpo_solve_voxel_fullcov(const float* xyz, int64_t n, const float* centre, double size, int G,
                            double lambda, double sf2, double sn2, int mean_mode,
                            int axis_override, int* axis_out, double* mean, double* cov)
{
    int axis = axis_override >= 0 ? axis_override : gpo_pca_axis(xyz, n, NULL, NULL);
    int p1, p2;
    param_axes(axis, &p1, &p2);
    *axis_out = axis;
    const int64_t Q = (int64_t)G * G;
    double* x1 = (double*)malloc(sizeof(double) * (size_t)n);
    double* x2 = (double*)malloc(sizeof(double) * (size_t)n);
    double* fm = (double*)malloc(sizeof(double) * (size_t)n);
    double* A = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* alpha = (double*)malloc(sizeof(double) * (size_t)n);
    double* k = (double*)malloc(sizeof(double) * (size_t)n);
    double* Z = (double*)malloc(sizeof(double) * (size_t)n * (size_t)Q);
    for (int64_t i = 0; i < n; ++i) {
        x1[i] = (double)xyz[3 * i + p1] - (double)centre[p1];
        x2[i] = (double)xyz[3 * i + p2] - (double)centre[p2];
        fm[i] = (double)xyz[3 * i + axis] - (double)centre[axis];
    }
    double m = 0.0;
    if (mean_mode == 1) {
        for (int64_t i = 0; i < n; ++i) m += fm[i];
        m /= (double)n;
    }
    for (int64_t i = 0; i < n; ++i) fm[i] -= m;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double d1 = x1[i] - x1[j], d2 = x2[i] - x2[j];
            A[i * n + j] = sf2 * exp(-lambda * (d1 * d1 + d2 * d2)) + (i == j ? sn2 : 0.0);
        }
    int status = GPO_OK;
    if (cholesky(A, n) != 0) {
        status = GPO_NOT_SPD;
        goto done;
    }
    forward_sub(A, n, fm, y);
    backward_sub(A, n, y, alpha);
    for (int64_t q = 0; q < Q; ++q) {
        double u = grid_node((int)(q / G), G, size), v = grid_node((int)(q % G), G, size);
        double mu = m;
        for (int64_t t = 0; t < n; ++t) {
            double d1 = x1[t] - u, d2 = x2[t] - v;
            k[t] = sf2 * exp(-lambda * (d1 * d1 + d2 * d2));
            mu += k[t] * alpha[t];
        }
        mean[q] = mu;
        forward_sub(A, n, k, Z + q * n);
    }
    for (int64_t q = 0; q < Q; ++q) {
        double u = grid_node((int)(q / G), G, size), v = grid_node((int)(q % G), G, size);
        for (int64_t r = 0; r < Q; ++r) {
            double u2 = grid_node((int)(r / G), G, size), v2 = grid_node((int)(r % G), G, size);
            double kk = sf2 * exp(-lambda * ((u - u2) * (u - u2) + (v - v2) * (v - v2)));
            double zz = 0.0;
            for (int64_t t = 0; t < n; ++t) zz += Z[q * n + t] * Z[r * n + t];
            cov[q * Q + r] = kk - zz;
        }
    }
done:
    free(x1); free(x2); free(fm); free(A); free(y); free(alpha); free(k); free(Z);
    return status;
}

/* ------------------------------------------------------------------ */
/* Structure similarity loss of Eq. 11: for every scan point P_j, the  */
/* minimum over all Gaussians k of |P_j - p_k| - mean(S_k), and the    */
/* mean of those minima over the points.  Brute force over k (ties:    */
/* the smallest k).  best[j], arg[j] per point; returns the mean.      */
/* ------------------------------------------------------------------ */
double gpo_structure_loss(const float* pts, int64_t n, const float* gpos, const float* gscale,
                          int64_t m, double* best, int64_t* arg)
{
    double total = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        double b = 0.0;
        int64_t bk = -1;
        for (int64_t k = 0; k < m; ++k) {
            double dx = (double)pts[3 * j] - (double)gpos[3 * k];
            double dy = (double)pts[3 * j + 1] - (double)gpos[3 * k + 1];
            double dz = (double)pts[3 * j + 2] - (double)gpos[3 * k + 2];
            double sbar = ((double)gscale[3 * k] + (double)gscale[3 * k + 1] + (double)gscale[3 * k + 2]) / 3.0;
            double v = sqrt(dx * dx + dy * dy + dz * dz) - sbar;
            if (bk < 0 || v < b) {
                b = v;
                bk = k;
            }
        }
        if (best) best[j] = b;
        if (arg) arg[j] = bk;
        total += b;
    }
    return n > 0 ? total / (double)n : 0.0;
}

/* ------------------------------------------------------------------ */
/* Alpha-blending rasterisation of 3D Gaussians (Sec. 3.3, Eq. 9): the */
/* colour C, depth D and silhouette S images of one pinhole camera.    */
/* Per Gaussian (FP64): t = Rc p + tc; culled when t_z <= near; 2D     */
/* mean u = fx t_x / t_z + cx, v = fy t_y / t_z + cy; covariance       */
/* Sigma = R diag(s^2) R^T (R from the unit quaternion), projected     */
/* Sigma' = J Rc Sigma Rc^T J^T + 0.3 I with the perspective Jacobian J */
/* at t (t_x / t_z, t_y / t_z clamped to 1.3 times the half field of   */
/* view); radius r = ceil(3 sqrt(lambda_max(Sigma'))).  A Gaussian     */
/* reaches pixel (x, y) (centre x + 1/2, y + 1/2) when the centre lies */
/* in [u - r, u + r] x [v - r, v + r]; there alpha = min(0.99, opacity */
/* exp(-d^T Sigma'^-1 d / 2)), skipped below 1/255.  Front to back by  */
/* depth (ties: smaller index): C += c alpha T, D += t_z alpha T,      */
/* S += alpha T, T *= 1 - alpha; blending stops before a Gaussian that */
/* would take T below 1e-4.  amb[pixel] = 1 when a decision at that    */
/* pixel lies within FP32 rounding of its threshold: bit 0 square      */
/* membership (1e-6 of |u| + |v| + r), bit 1 the radius rounding (3     */
/* sqrt(lambda_max) within 1e-5 of an integer, pixels within 1 of the  */
/* edge), bit 2 the 1/255 cut and bit 3 the 1e-4 stop (1e-5 relative). */
/* The depth that orders and culls is computed in FP32 as the kernel   */
/* does (same operations, same order, each rounded), so those decisions */
/* match exactly.                                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    double u, v, z, ca, cb, cc, r, op, col[3];
    float zkey;
    int ok, amb_r;
} gpo_splat;

typedef struct {
    double z;
    int64_t k;
} gpo_zk;

static int cmp_zk(const void* a, const void* b)
{
    const gpo_zk* x = (const gpo_zk*)a;
    const gpo_zk* y = (const gpo_zk*)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return x->k < y->k ? -1 : (x->k > y->k ? 1 : 0);
}

void gpo_rasterize(const float* pos, const float* scale, const float* quat, const float* opac,
                   const float* color, int64_t m, const double* Rc, const double* tc, double fx,
                   double fy, double cx, double cy, int W, int H, double near, double* C,
                   double* D, double* S, uint8_t* amb)
{
    gpo_splat* g = (gpo_splat*)malloc(sizeof(gpo_splat) * (size_t)(m > 0 ? m : 1));
    const double limx = 1.3 * (double)W / (2.0 * fx), limy = 1.3 * (double)H / (2.0 * fy);
    for (int64_t k = 0; k < m; ++k) {
        gpo_splat* q = &g[k];
        q->ok = 0;
        q->amb_r = 0;
        double t[3];
        for (int a = 0; a < 3; ++a)
            t[a] = Rc[3 * a] * pos[3 * k] + Rc[3 * a + 1] * pos[3 * k + 1] + Rc[3 * a + 2] * pos[3 * k + 2] + tc[a];
        /* the depth that orders and culls: FP32, rounded after each operation in this
           order, so the kernel takes the same decisions (its inputs are FP32) */
        const float zk = (((float)Rc[6] * pos[3 * k]) + ((float)Rc[7] * pos[3 * k + 1])) +
                         ((float)Rc[8] * pos[3 * k + 2]) + (float)tc[2];
        q->zkey = zk;
        if (!(zk > (float)near)) continue;
        double qw = quat[4 * k], qx = quat[4 * k + 1], qy = quat[4 * k + 2], qz = quat[4 * k + 3];
        double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= qn; qx /= qn; qy /= qn; qz /= qn;
        double R[3][3] = {
            {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy)},
            {2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx)},
            {2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)}};
        double Sg[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int c = 0; c < 3; ++c) acc += R[a][c] * (double)scale[3 * k + c] * (double)scale[3 * k + c] * R[b][c];
                Sg[a][b] = acc;
            }
        double xz = t[0] / t[2], yz = t[1] / t[2];
        if (xz < -limx) xz = -limx;
        if (xz > limx) xz = limx;
        if (yz < -limy) yz = -limy;
        if (yz > limy) yz = limy;
        double J[2][3] = {{fx / t[2], 0.0, -fx * xz / t[2]}, {0.0, fy / t[2], -fy * yz / t[2]}};
        double T2[2][3];  /* J Rc */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int c = 0; c < 3; ++c) acc += J[a][c] * Rc[3 * c + b];
                T2[a][b] = acc;
            }
        double P2[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0.0;
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) acc += T2[a][c] * Sg[c][d] * T2[b][d];
                P2[a][b] = acc;
            }
        double sa = P2[0][0] + 0.3, sb = P2[0][1], sc = P2[1][1] + 0.3;
        double det = sa * sc - sb * sb;
        if (!(det > 0.0)) continue;
        double mid = 0.5 * (sa + sc);
        double disc = mid * mid - det;
        double lmax = mid + sqrt(disc > 0.1 ? disc : 0.1);
        double r3 = 3.0 * sqrt(lmax);
        q->r = ceil(r3);
        q->amb_r = fabs(r3 - floor(r3 + 0.5)) < 1e-5 * r3;
        q->ca = sc / det;
        q->cb = -sb / det;
        q->cc = sa / det;
        q->u = fx * t[0] / t[2] + cx;
        q->v = fy * t[1] / t[2] + cy;
        q->z = t[2];
        q->op = opac[k];
        for (int a = 0; a < 3; ++a) q->col[a] = color[3 * k + a];
        q->ok = 1;
    }
    gpo_zk* list = (gpo_zk*)malloc(sizeof(gpo_zk) * (size_t)(m > 0 ? m : 1));
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double px = x + 0.5, py = y + 0.5;
            const int64_t o = (int64_t)y * W + x;
            int a_flag = 0;
            int64_t cnt = 0;
            for (int64_t k = 0; k < m; ++k) {
                const gpo_splat* q = &g[k];
                if (!q->ok) continue;
                const double ex = fabs(px - q->u), ey = fabs(py - q->v);
                const double e = ex > ey ? ex : ey;
                if (e <= q->r + 1.0 && e >= q->r - 1.0) {
                    /* the square's edge matters only where the Gaussian would be drawn */
                    const double dx = px - q->u, dy = py - q->v;
                    const double pw = -0.5 * (q->ca * dx * dx + q->cc * dy * dy) - q->cb * dx * dy;
                    if (q->op * exp(pw) >= (1.0 - 1e-5) / 255.0) {
                        if (fabs(e - q->r) < 1e-6 * (fabs(q->u) + fabs(q->v) + q->r + 1.0)) a_flag |= 1;
                        if (q->amb_r) a_flag |= 2;
                    }
                }
                if (e > q->r) continue;
                list[cnt].z = (double)q->zkey;
                list[cnt].k = k;
                ++cnt;
            }
            qsort(list, (size_t)cnt, sizeof(gpo_zk), cmp_zk);
            double T = 1.0, c3[3] = {0, 0, 0}, dd = 0.0, ss = 0.0;
            for (int64_t i = 0; i < cnt; ++i) {
                const gpo_splat* q = &g[list[i].k];
                const double dx = px - q->u, dy = py - q->v;
                const double power = -0.5 * (q->ca * dx * dx + q->cc * dy * dy) - q->cb * dx * dy;
                double alpha = q->op * exp(power);
                if (alpha > 0.99) alpha = 0.99;
                if (fabs(alpha - 1.0 / 255.0) < 1e-5 / 255.0) a_flag |= 4;
                if (alpha < 1.0 / 255.0) continue;
                const double nt = T * (1.0 - alpha);
                if (fabs(nt - 1e-4) < 1e-9) a_flag |= 8;
                if (nt < 1e-4) break;
                for (int a = 0; a < 3; ++a) c3[a] += q->col[a] * alpha * T;
                dd += q->z * alpha * T;
                ss += alpha * T;
                T = nt;
            }
            for (int a = 0; a < 3; ++a) C[3 * o + a] = c3[a];
            D[o] = dd;
            S[o] = ss;
            if (amb) amb[o] = (uint8_t)a_flag;
        }
    free(list);
    free(g);
}

/* ------------------------------------------------------------------ */
/* Quaternion (w, x, y, z) of a proper rotation matrix R (row-major), */
/* the textbook trace/major-diagonal branches; sign fixed to w >= 0.  */
/* ------------------------------------------------------------------ */
static void quat_from_rot(const double R[3][3], double q[4])
{
    double tr = R[0][0] + R[1][1] + R[2][2];
    double w, x, y, z;
    if (tr > 0.0) {
        double S = sqrt(tr + 1.0) * 2.0;
        w = 0.25 * S;
        x = (R[2][1] - R[1][2]) / S;
        y = (R[0][2] - R[2][0]) / S;
        z = (R[1][0] - R[0][1]) / S;
    } else if (R[0][0] > R[1][1] && R[0][0] > R[2][2]) {
        double S = sqrt(1.0 + R[0][0] - R[1][1] - R[2][2]) * 2.0;
        w = (R[2][1] - R[1][2]) / S;
        x = 0.25 * S;
        y = (R[0][1] + R[1][0]) / S;
        z = (R[0][2] + R[2][0]) / S;
    } else if (R[1][1] > R[2][2]) {
        double S = sqrt(1.0 + R[1][1] - R[0][0] - R[2][2]) * 2.0;
        w = (R[0][2] - R[2][0]) / S;
        x = (R[0][1] + R[1][0]) / S;
        y = 0.25 * S;
        z = (R[1][2] + R[2][1]) / S;
    } else {
        double S = sqrt(1.0 + R[2][2] - R[0][0] - R[1][1]) * 2.0;
        w = (R[1][0] - R[0][1]) / S;
        x = (R[0][2] + R[2][0]) / S;
        y = (R[1][2] + R[2][1]) / S;
        z = 0.25 * S;
    }
    double nq = sqrt(w * w + x * x + y * y + z * z);
    double sgn = (w < 0.0) ? -1.0 : 1.0;
    q[0] = sgn * w / nq; q[1] = sgn * x / nq; q[2] = sgn * y / nq; q[3] = sgn * z / nq;
}

/* Canonical sign of an eigenvector: its largest-magnitude component is   */
/* made positive (ties go to the lower index).                           */
static void canon_sign(double e[3])
{
    int kmax = 0;
    for (int k = 1; k < 3; ++k)
        if (fabs(e[k]) > fabs(e[kmax])) kmax = k;
    if (e[kmax] < 0.0)
        for (int k = 0; k < 3; ++k) e[k] = -e[k];
}

/* ------------------------------------------------------------------ */
/* Gaussian initialisation of one voxel (Sec. 3.2, Eq. 6-8).          */
/*                                                                    */
/* mean/var: the voxel's G*G GPR outputs (voxel-local value coord.);  */
/* G = n_s * n_r; subgrid beta = (bi, bj) is the n_r x n_r block of   */
/* query nodes starting at (bi*n_r, bj*n_r), Gaussian index           */
/* bi*n_s + bj.  Outputs per Gaussian: pos (world, [3]), scale ([3],  */
/* descending), quat ([4], w x y z); also the raw Phi ([9]) if given. */
/* ------------------------------------------------------------------ */
int gpo_init_voxel(const double* mean, const double* var, int axis, const float* centre,
                   double size, int G, int n_s, int n_r, double sf2, int init_mode,
                   double* pos, double* scale, double* quat, double* phi_out)
{
    int p1, p2;
    if (n_r < 1 || n_r > 8 || n_s * n_r != G || axis < 0 || axis > 2) return -1;
    param_axes(axis, &p1, &p2);
    const double v_floor = 1e-6 * sf2;
    const double s_floor = 1e-4 * size;
    for (int bi = 0; bi < n_s; ++bi)
        for (int bj = 0; bj < n_s; ++bj) {
            int g = bi * n_s + bj;
            double P[64][3], w[64];
            int cnt = 0;
            for (int ii = 0; ii < n_r; ++ii)
                for (int jj = 0; jj < n_r; ++jj) {
                    int i = bi * n_r + ii, j = bj * n_r + jj;
                    int q = i * G + j;
                    P[cnt][p1] = grid_node(i, G, size);
                    P[cnt][p2] = grid_node(j, G, size);
                    P[cnt][axis] = mean[q];
                    w[cnt] = 1.0 / (var[q] > v_floor ? var[q] : v_floor);
                    ++cnt;
                }
            /* Eq. 6: weighted position */
            double sw = 0.0, p[3] = {0, 0, 0};
            for (int t = 0; t < cnt; ++t) {
                sw += w[t];
                for (int k = 0; k < 3; ++k) p[k] += w[t] * P[t][k];
            }
            for (int k = 0; k < 3; ++k) p[k] /= sw;
            /* Eq. 7: Phi = Q^T diag(w) Q / sum w,  Q = P - p */
            double Phi[3][3] = {{0}};
            for (int t = 0; t < cnt; ++t) {
                double Q[3];
                for (int k = 0; k < 3; ++k) Q[k] = P[t][k] - p[k];
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) Phi[r][c] += w[t] * Q[r] * Q[c];
            }
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) Phi[r][c] /= sw;
            if (phi_out)
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) phi_out[9 * g + 3 * r + c] = Phi[r][c];

            for (int k = 0; k < 3; ++k) pos[3 * g + k] = (double)centre[k] + p[k];

            if (init_mode == 1) {
                /* Eq. 8 as printed: S = diag(Phi), R = identity quaternion */
                for (int k = 0; k < 3; ++k) scale[3 * g + k] = Phi[k][k];
                quat[4 * g + 0] = 1.0; quat[4 * g + 1] = 0.0;
                quat[4 * g + 2] = 0.0; quat[4 * g + 3] = 0.0;
                continue;
            }
            /* Eq. 5 read backwards: Phi = R S S^T R^T, S = sqrt(eigenvalues) */
            double ev[3], V[3][3];
            jacobi3(Phi, ev, V);
            int idx[3] = {0, 1, 2};
            for (int a = 0; a < 3; ++a) /* sort descending */
                for (int b = a + 1; b < 3; ++b)
                    if (ev[idx[b]] > ev[idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
            double e1[3], e2[3], e3[3];
            for (int k = 0; k < 3; ++k) { e1[k] = V[k][idx[0]]; e2[k] = V[k][idx[1]]; }
            canon_sign(e1);
            canon_sign(e2);
            e3[0] = e1[1] * e2[2] - e1[2] * e2[1];
            e3[1] = e1[2] * e2[0] - e1[0] * e2[2];
            e3[2] = e1[0] * e2[1] - e1[1] * e2[0];
            double R[3][3];
            for (int k = 0; k < 3; ++k) { R[k][0] = e1[k]; R[k][1] = e2[k]; R[k][2] = e3[k]; }
            for (int a = 0; a < 3; ++a) {
                double l = ev[idx[a]];
                scale[3 * g + a] = sqrt(l > s_floor * s_floor ? l : s_floor * s_floor);
            }
            quat_from_rot(R, &quat[4 * g]);
        }
    return GPO_OK;
}

/* ------------------------------------------------------------------ */
/* Batched drivers.  Voxels are independent, so worker threads take   */
/* one voxel at a time from a shared counter; no arithmetic changes.  */
/* ------------------------------------------------------------------ */
typedef struct {
    const float* xyz;
    const int64_t* offsets;
    int64_t nvox;
    const float* centres;
    const float* lambda;
    const float* sf2;
    const float* sn2;
    double size;
    int G, tau, mean_mode;
    const int32_t* axis_override;
    int32_t* axis;
    double* mean;
    double* var;
    int32_t* status;
    int64_t next;
} batch_job;

static void* batch_worker(void* arg)
{
    batch_job* J = (batch_job*)arg;
    const int64_t GG = (int64_t)J->G * J->G;
    for (;;) {
        int64_t v = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (v >= J->nvox) break;
        int64_t b = J->offsets[v], n = J->offsets[v + 1] - b;
        double* mu = J->mean + v * GG;
        double* va = J->var + v * GG;
        if (n < J->tau || n <= 0) {
            J->status[v] = GPO_BELOW_TAU;
            J->axis[v] = -1;
            for (int64_t q = 0; q < GG; ++q) { mu[q] = 0.0; va[q] = (double)J->sf2[v]; }
            continue;
        }
        int ax = 0;
        int ov = J->axis_override ? J->axis_override[v] : -1;
        J->status[v] = gpo_solve_voxel(J->xyz + 3 * b, n, J->centres + 3 * v, J->size, J->G,
                                       (double)J->lambda[v], (double)J->sf2[v],
                                       (double)J->sn2[v], J->mean_mode, ov, &ax, mu, va);
        J->axis[v] = ax;
    }
    return NULL;
}

int gpo_solve_batch(const float* xyz, const int64_t* offsets, int64_t nvox, const float* centres,
                    const float* lambda, const float* sf2, const float* sn2, double size, int G,
                    int tau, int mean_mode, const int32_t* axis_override, int nthreads,
                    int32_t* axis, double* mean, double* var, int32_t* status)
{
    batch_job J = {xyz, offsets, nvox, centres, lambda, sf2, sn2, size, G, tau, mean_mode,
                   axis_override, axis, mean, var, status, 0};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, batch_worker, &J);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    return GPO_OK;
}

int gpo_init_batch(const double* mean, const double* var, const int32_t* axis,
                   const float* centres, const float* sf2, int64_t nvox, double size, int G,
                   int n_s, int n_r, int init_mode, double* pos, double* scale, double* quat)
{
    const int64_t GG = (int64_t)G * G, NG = (int64_t)n_s * n_s;
    for (int64_t v = 0; v < nvox; ++v) {
        if (axis[v] < 0) { /* below tau: no Gaussians are initialised */
            for (int64_t g = 0; g < NG; ++g) {
                for (int k = 0; k < 3; ++k) {
                    pos[3 * (v * NG + g) + k] = (double)centres[3 * v + k];
                    scale[3 * (v * NG + g) + k] = 0.0;
                }
                quat[4 * (v * NG + g) + 0] = 1.0;
                quat[4 * (v * NG + g) + 1] = 0.0;
                quat[4 * (v * NG + g) + 2] = 0.0;
                quat[4 * (v * NG + g) + 3] = 0.0;
            }
            continue;
        }
        gpo_init_voxel(mean + v * GG, var + v * GG, axis[v], centres + 3 * v, size, G, n_s, n_r,
                       (double)sf2[v], init_mode, pos + 3 * v * NG, scale + 3 * v * NG,
                       quat + 4 * v * NG, NULL);
    }
    return GPO_OK;
}
