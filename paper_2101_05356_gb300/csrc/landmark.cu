// Sparse landmark loss of Sec. 4, Eq. (landmark):
//     E_land = sum_l || Pi(Gamma(v_{i_l})) - z_l ||^2
// over L landmark vertices i_l of the morphed face (v = a_s + Sigma coef,
// Sec. 3.1), posed by Gamma(v) = R^T (v - T) with R = Rz Ry Rx and projected
// by the pinhole Pi (principal point at the image centre, image y down), and
// its gradient with respect to the coefficients, the Euler angles, T and the
// focal length.  One block per call, one thread per landmark, all in FP64
// (L <= 256 vertices: the cost is negligible next to a render), with sums in a
// fixed order so results are reproducible.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int LM_THREADS = 256;

__global__ void __launch_bounds__(LM_THREADS) k_landmarks(LandmarkArgs a) {
    __shared__ double R[9], D[3][9];
    __shared__ double gv[LM_THREADS][3];          // dE/dv (model space) per landmark
    __shared__ double red[LM_THREADS][8];         // e, dT[3], dtheta[3], df per landmark
    const int l = threadIdx.x;
    if (l == 0) {
        const double p = a.rot[0], q = a.rot[1], r = a.rot[2];
        const double sx = sin(p), cx = cos(p), sy = sin(q), cy = cos(q), sz = sin(r), cz = cos(r);
        const double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx}, dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
        const double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy}, dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
        const double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1}, dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
        auto mul = [](const double* A, const double* B, double* C) {
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
                    C[3 * i + j] = s;
                }
        };
        double t[9];
        mul(Ry, Rx, t); mul(Rz, t, R);
        mul(Ry, dRx, t); mul(Rz, t, D[0]);
        mul(dRy, Rx, t); mul(Rz, t, D[1]);
        mul(Ry, Rx, t); mul(dRz, t, D[2]);
    }
    __syncthreads();
    double loc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    gv[l][0] = gv[l][1] = gv[l][2] = 0.0;
    if (l < a.L) {
        const int i = a.idx[l];
        double v[3];
        for (int c = 0; c < 3; ++c) {
            double s = a.mean[3 * i + c];
            for (int k = 0; k < a.K; ++k) s += (double)a.coef[k] * (double)a.basis[(size_t)k * a.ld + 3 * i + c];
            v[c] = s;
        }
        const double w[3] = {v[0] - a.trans[0], v[1] - a.trans[1], v[2] - a.trans[2]};
        double vp[3];                                   // v' = R^T w
        for (int c = 0; c < 3; ++c) vp[c] = R[c] * w[0] + R[3 + c] * w[1] + R[6 + c] * w[2];
        const double f = a.focal[0], iz = 1.0 / vp[2];
        const double x = 0.5 * a.W - f * vp[0] * iz, y = 0.5 * a.H + f * vp[1] * iz;
        if (a.proj) {
            a.proj[2 * l] = (float)x;
            a.proj[2 * l + 1] = (float)y;
        }
        const double rx = x - a.z[2 * l], ry = y - a.z[2 * l + 1];
        loc[0] = rx * rx + ry * ry;
        const double ex = 2.0 * rx, ey = 2.0 * ry;      // dE/dx, dE/dy
        const double gp[3] = {-ex * f * iz, ey * f * iz, ex * f * vp[0] * iz * iz - ey * f * vp[1] * iz * iz};
        loc[7] = -ex * vp[0] * iz + ey * vp[1] * iz;    // dE/df
        for (int j = 0; j < 3; ++j) {                    // dE/dw = R g'
            const double gw = R[3 * j] * gp[0] + R[3 * j + 1] * gp[1] + R[3 * j + 2] * gp[2];
            gv[l][j] = gw;
            loc[1 + j] = -gw;                            // dE/dT
        }
        for (int q = 0; q < 3; ++q) {                    // dv'_c / dtheta_q = sum_j D_q[j][c] w_j
            double s = 0.0;
            for (int c = 0; c < 3; ++c) s += gp[c] * (D[q][c] * w[0] + D[q][3 + c] * w[1] + D[q][6 + c] * w[2]);
            loc[4 + q] = s;
        }
    }
    for (int k = 0; k < 8; ++k) red[l][k] = loc[k];
    __syncthreads();
    if (l < 8) {                                         // landmark order
        double s = 0.0;
        for (int m = 0; m < a.L; ++m) s += red[m][l];
        s *= (double)a.weight;
        if (l == 0) *a.loss = s;
        else if (l < 4) { if (a.g_trans) a.g_trans[l - 1] += (float)s; }
        else if (l < 7) { if (a.g_rot) a.g_rot[l - 4] += (float)s; }
        else if (a.g_focal) a.g_focal[0] += (float)s;
    }
    if (a.g_coef)
        for (int k = l; k < a.K; k += LM_THREADS) {      // dE/dcoef_k = sum_l basis_k(v_l) . dE/dv_l
            double s = 0.0;
            for (int m = 0; m < a.L; ++m) {
                const int i = a.idx[m];
                const float* b = a.basis + (size_t)k * a.ld + 3 * i;
                s += (double)b[0] * gv[m][0] + (double)b[1] * gv[m][1] + (double)b[2] * gv[m][2];
            }
            a.g_coef[k] += (float)(s * (double)a.weight);
        }
}

}  // namespace

void launch_landmarks(const LandmarkArgs& a, cudaStream_t st) {
    k_landmarks<<<1, LM_THREADS, 0, st>>>(a);
    fr_count_launches(1);
}
