// Derivatives of the unnormalised ACA homography with respect to the target
// points (the source is held fixed), for networks that regress 4-point
// offsets (Sec. 5.3: ACA uses only +, -, * and is naturally
// differentiable).  Both kernels evaluate the vector-Jacobian product
// grad_tgt = (dH/dtgt)^T grad_H by reverse-mode differentiation of the
// chain, written out by hand:
//
//   general source (Eq. 24): H = A * X, A = H_A2^-1 (Eq. 22), X = H_C H_A1,
//     dA = G X^T, dX = A^T G, dH_C = dX H_A1^T, then Eq. 28-29 and Eq. 21/25/27
//     back to the target vectors M2N2, M2P2, M2Q2 and the point M2;
//   rectangle source (Eq. 42): H = A * B with A = [[N2 P2 M2];[1 1 1]],
//     dA = G B^T, dB = A^T G, then Q4, t2 (Eq. 25, 27) back to the corners.
//
// Each set is 25 (general) or 17 (rectangle) floats in and 8 out, a stream:
// four adjacent sets per thread with float4 SoA loads, like the solvers.
#include "aca_math.cuh"
#include "common.cuh"
#include "pdl.cuh"  // launched as programmatic dependents, as the forward kernels (solve.cu)

namespace aca {

// dL/d(Q4x, Q4y, fA2 via t2) -> dL/d(target corners); shared tail of both
// products.  gMN/gMP/gM2 carry the direct contributions already collected.
ACA_HD void back_target_crosses(float gQ4x, float gQ4y, float gt2, float MN2x, float MN2y, float MP2x, float MP2y,
                                float MQ2x, float MQ2y, float gMN2x, float gMN2y, float gMP2x, float gMP2y,
                                float gM2x, float gM2y, float g[8])
{
    // t2 = fA2 - Q4x - Q4y (Eq. 27)
    const float gfA2 = gt2;
    const float gQx = F_SUB(gQ4x, gt2), gQy = F_SUB(gQ4y, gt2);
    // fA2 = MN2 x MP2 (Eq. 21); Q4x = MQ2 x MP2, Q4y = MN2 x MQ2 (Eq. 25)
    gMN2x = F_FMA(gfA2, MP2y, F_FMA(gQy, MQ2y, gMN2x));
    gMN2y = F_SUB(gMN2y, F_FMA(gfA2, MP2x, F_MUL(gQy, MQ2x)));
    gMP2x = F_SUB(gMP2x, F_FMA(gfA2, MN2y, F_MUL(gQx, MQ2y)));
    gMP2y = F_FMA(gfA2, MN2x, F_FMA(gQx, MQ2x, gMP2y));
    const float gMQ2x = F_SUB(F_MUL(gQx, MP2y), F_MUL(gQy, MN2y));
    const float gMQ2y = F_SUB(F_MUL(gQy, MN2x), F_MUL(gQx, MP2x));
    // MN2 = N2 - M2, MP2 = P2 - M2, MQ2 = Q2 - M2
    g[0] = F_SUB(gM2x, F_ADD(F_ADD(gMN2x, gMP2x), gMQ2x));
    g[1] = F_SUB(gM2y, F_ADD(F_ADD(gMN2y, gMP2y), gMQ2y));
    g[2] = gMN2x;
    g[3] = gMN2y;
    g[4] = gMP2x;
    g[5] = gMP2y;
    g[6] = gMQ2x;
    g[7] = gMQ2y;
}

ACA_HD void aca_vjp(const Set &s, const float G[9], float g[8])
{
    AcaParts p;
    aca_parts(s, p);
    const float c11 = F_MUL(F_MUL(p.t1, p.Q3y), p.Q4x);
    const float c22 = F_MUL(F_MUL(p.t1, p.Q3x), p.Q4y);
    const float c33 = F_MUL(F_MUL(p.t2, p.Q3x), p.Q3y);
    // H_A1 = L1 T(-M1) (Eq. 20)
    const float A1[9] = {p.MP1y, -p.MP1x, F_SUB(F_MUL(p.MP1x, s.M1y), F_MUL(p.MP1y, s.M1x)),
                         -p.MN1y, p.MN1x, F_SUB(F_MUL(p.MN1y, s.M1x), F_MUL(p.MN1x, s.M1y)),
                         0.0f, 0.0f, p.fA1};
    // X = H_C H_A1 with H_C = [[c11,0,0],[0,c22,0],[c11-c33, c22-c33, c33]]
    float X[9];
    for (int j = 0; j < 3; ++j) {
        X[j] = F_MUL(c11, A1[j]);
        X[3 + j] = F_MUL(c22, A1[3 + j]);
        X[6 + j] = F_FMA(F_SUB(c11, c33), A1[j], F_FMA(F_SUB(c22, c33), A1[3 + j], F_MUL(c33, A1[6 + j])));
    }
    // dA = G X^T for A = [[MN2x, MP2x, M2x], [MN2y, MP2y, M2y], [0, 0, 1]]
    float gA[6];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k)
            gA[3 * i + k] = F_FMA(G[3 * i], X[3 * k], F_FMA(G[3 * i + 1], X[3 * k + 1], F_MUL(G[3 * i + 2], X[3 * k + 2])));
    // dX = A^T G
    float gX[9];
    for (int j = 0; j < 3; ++j) {
        gX[j] = F_FMA(p.MN2x, G[j], F_MUL(p.MN2y, G[3 + j]));
        gX[3 + j] = F_FMA(p.MP2x, G[j], F_MUL(p.MP2y, G[3 + j]));
        gX[6 + j] = F_FMA(s.M2x, G[j], F_FMA(s.M2y, G[3 + j], G[6 + j]));
    }
    // dH_C = dX H_A1^T (only the entries H_C depends on)
    auto dC = [&](int i, int k) {
        return F_FMA(gX[3 * i], A1[3 * k], F_FMA(gX[3 * i + 1], A1[3 * k + 1], F_MUL(gX[3 * i + 2], A1[3 * k + 2])));
    };
    const float gC00 = dC(0, 0), gC11 = dC(1, 1), gC20 = dC(2, 0), gC21 = dC(2, 1), gC22 = dC(2, 2);
    // Eq. 28: c11 enters (0,0) and (2,0); c22 enters (1,1) and (2,1); c33 enters (2,0), (2,1) negatively and (2,2)
    const float gc11 = F_ADD(gC00, gC20);
    const float gc22 = F_ADD(gC11, gC21);
    const float gc33 = F_SUB(gC22, F_ADD(gC20, gC21));
    // Eq. 29
    const float gQ4x = F_MUL(gc11, F_MUL(p.t1, p.Q3y));
    const float gQ4y = F_MUL(gc22, F_MUL(p.t1, p.Q3x));
    const float gt2 = F_MUL(gc33, F_MUL(p.Q3x, p.Q3y));
    back_target_crosses(gQ4x, gQ4y, gt2, p.MN2x, p.MN2y, p.MP2x, p.MP2y, p.MQ2x, p.MQ2y, gA[0], gA[3], gA[1], gA[4],
                        gA[2], gA[5], g);
}

ACA_HD void rect_vjp(const float t[8], const Rect &R, const float G[9], float g[8])
{
    RectParts p;
    rect_parts(t, p);
    const float k = F_ADD(F_FMA(R.r, R.y0, R.x0), R.w);
    // B of Eq. 42
    const float B[9] = {p.Q4x, 0.0f, -F_MUL(p.Q4x, R.x0),
                        0.0f, F_MUL(R.r, p.Q4y), -F_MUL(F_MUL(R.r, p.Q4y), R.y0),
                        p.t2, F_MUL(R.r, p.t2), -F_MUL(p.t2, k)};
    // dA = G B^T for A = [[N2x, P2x, M2x], [N2y, P2y, M2y], [1, 1, 1]]
    float gA[6];
    for (int i = 0; i < 2; ++i)
        for (int c = 0; c < 3; ++c)
            gA[3 * i + c] = F_FMA(G[3 * i], B[3 * c], F_FMA(G[3 * i + 1], B[3 * c + 1], F_MUL(G[3 * i + 2], B[3 * c + 2])));
    // dB = A^T G, only the entries B depends on
    const float A[9] = {t[2], t[4], t[0], t[3], t[5], t[1], 1.0f, 1.0f, 1.0f};
    auto dB = [&](int r, int c) {
        return F_FMA(A[r], G[c], F_FMA(A[3 + r], G[3 + c], F_MUL(A[6 + r], G[6 + c])));
    };
    const float gQ4x = F_FMA(-R.x0, dB(0, 2), dB(0, 0));
    const float gQ4y = F_MUL(R.r, F_FMA(-R.y0, dB(1, 2), dB(1, 1)));
    const float gt2 = F_FMA(-k, dB(2, 2), F_FMA(R.r, dB(2, 1), dB(2, 0)));
    // direct A contributions: column 0 = N2, column 1 = P2, column 2 = M2
    back_target_crosses(gQ4x, gQ4y, gt2, p.MN2x, p.MN2y, p.MP2x, p.MP2y, p.MQ2x, p.MQ2y, 0.0f, 0.0f, 0.0f, 0.0f,
                        gA[2], gA[5], g);
    g[2] = F_ADD(g[2], gA[0]);
    g[3] = F_ADD(g[3], gA[3]);
    g[4] = F_ADD(g[4], gA[1]);
    g[5] = F_ADD(g[5], gA[4]);
}

__global__ void __launch_bounds__(256) aca_backward_vec4_kernel(const float *__restrict__ pts,
                                                                 const float *__restrict__ gH,
                                                                 float *__restrict__ gT, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    const int64_t nq = (n + 3) >> 2, ldq = ld >> 2;
    const float4 *in = reinterpret_cast<const float4 *>(pts);
    const float4 *gin = reinterpret_cast<const float4 *>(gH);
    float4 *out = reinterpret_cast<float4 *>(gT);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        float4 v[16], gv[9], o[8];
#pragma unroll
        for (int k = 0; k < 16; ++k)
            v[k] = ld_stream(in + k * ldq + q);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            gv[k] = ld_stream(gin + k * ldq + q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Set s;
            float *sv = &s.M1x;
            float G[9], g[8];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                sv[k] = (&v[k].x)[j];
#pragma unroll
            for (int k = 0; k < 9; ++k)
                G[k] = (&gv[k].x)[j];
            aca_vjp(s, G, g);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                (&o[k].x)[j] = g[k];
        }
        const int64_t i0 = q << 2;
        if (i0 + 3 < n) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                st_stream(out + k * ldq + q, o[k]);
        } else {
            for (int j = 0; j < 4 && i0 + j < n; ++j)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    gT[k * ld + i0 + j] = (&o[k].x)[j];
        }
    }
}

__global__ void __launch_bounds__(256) aca_backward_scalar_kernel(const float *__restrict__ pts,
                                                                   const float *__restrict__ gH,
                                                                   float *__restrict__ gT, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Set s;
        float *sv = &s.M1x;
        float G[9], g[8];
#pragma unroll
        for (int k = 0; k < 16; ++k)
            sv[k] = ld_stream(pts + k * ld + i);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            G[k] = ld_stream(gH + k * ld + i);
        aca_vjp(s, G, g);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            st_stream(gT + k * ld + i, g[k]);
    }
}

__global__ void __launch_bounds__(256) rect_backward_vec4_kernel(const float *__restrict__ tgt, Rect R,
                                                                  const float *__restrict__ gH,
                                                                  float *__restrict__ gT, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    const int64_t nq = (n + 3) >> 2, ldq = ld >> 2;
    const float4 *in = reinterpret_cast<const float4 *>(tgt);
    const float4 *gin = reinterpret_cast<const float4 *>(gH);
    float4 *out = reinterpret_cast<float4 *>(gT);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        float4 v[8], gv[9], o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = ld_stream(in + k * ldq + q);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            gv[k] = ld_stream(gin + k * ldq + q);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float t[8], G[9], g[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                t[k] = (&v[k].x)[j];
#pragma unroll
            for (int k = 0; k < 9; ++k)
                G[k] = (&gv[k].x)[j];
            rect_vjp(t, R, G, g);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                (&o[k].x)[j] = g[k];
        }
        const int64_t i0 = q << 2;
        if (i0 + 3 < n) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                st_stream(out + k * ldq + q, o[k]);
        } else {
            for (int j = 0; j < 4 && i0 + j < n; ++j)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    gT[k * ld + i0 + j] = (&o[k].x)[j];
        }
    }
}

__global__ void __launch_bounds__(256) rect_backward_scalar_kernel(const float *__restrict__ tgt, Rect R,
                                                                    const float *__restrict__ gH,
                                                                    float *__restrict__ gT, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float t[8], G[9], g[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            t[k] = ld_stream(tgt + k * ld + i);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            G[k] = ld_stream(gH + k * ld + i);
        rect_vjp(t, R, G, g);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            st_stream(gT + k * ld + i, g[k]);
    }
}

}  // namespace aca

using namespace aca;

extern "C" aca_status aca_backward(const float *pts, const float *grad_H, float *grad_tgt, int64_t n, int64_t ld,
                                   void *stream)
{
    if (n < 0 || ld < n)
        return set_error(ACA_ERR_INVALID_ARG, "aca_backward: need 0 <= n <= ld");
    if (n == 0)
        return ACA_OK;
    if (!pts || !grad_H || !grad_tgt)
        return set_error(ACA_ERR_INVALID_ARG, "aca_backward: null pointer");
    const cudaStream_t st = as_stream(stream);
    const int threads = 256;
    if (n >= kSmallBatch && ld % 4 == 0 && aligned16(pts) && aligned16(grad_H) && aligned16(grad_tgt)) {
        const int grid = resident_grid(aca_backward_vec4_kernel, threads, 0, ((n + 3) / 4 + threads - 1) / threads);
        launch_after_previous(aca_backward_vec4_kernel, dim3(grid), dim3(threads), 0, st, pts, grad_H, grad_tgt, n,
                              ld);
    } else {
        const int grid = resident_grid(aca_backward_scalar_kernel, threads, 0, (n + threads - 1) / threads);
        launch_after_previous(aca_backward_scalar_kernel, dim3(grid), dim3(threads), 0, st, pts, grad_H, grad_tgt, n,
                              ld);
    }
    return check_launch("aca_backward");
}

extern "C" aca_status aca_rect_backward(const float *tgt, float x0, float y0, float w, float r, const float *grad_H,
                                        float *grad_tgt, int64_t n, int64_t ld, void *stream)
{
    if (n < 0 || ld < n)
        return set_error(ACA_ERR_INVALID_ARG, "aca_rect_backward: need 0 <= n <= ld");
    if (!(w > 0) || !(r > 0))
        return set_error(ACA_ERR_INVALID_ARG, "aca_rect_backward: width and aspect ratio must be > 0");
    if (n == 0)
        return ACA_OK;
    if (!tgt || !grad_H || !grad_tgt)
        return set_error(ACA_ERR_INVALID_ARG, "aca_rect_backward: null pointer");
    const Rect R{x0, y0, w, r};
    const cudaStream_t st = as_stream(stream);
    const int threads = 256;
    if (n >= kSmallBatch && ld % 4 == 0 && aligned16(tgt) && aligned16(grad_H) && aligned16(grad_tgt)) {
        const int grid = resident_grid(rect_backward_vec4_kernel, threads, 0, ((n + 3) / 4 + threads - 1) / threads);
        launch_after_previous(rect_backward_vec4_kernel, dim3(grid), dim3(threads), 0, st, tgt, R, grad_H,
                              grad_tgt, n, ld);
    } else {
        const int grid = resident_grid(rect_backward_scalar_kernel, threads, 0, (n + threads - 1) / threads);
        launch_after_previous(rect_backward_scalar_kernel, dim3(grid), dim3(threads), 0, st, tgt, R, grad_H,
                              grad_tgt, n, ld);
    }
    return check_launch("aca_rect_backward");
}
