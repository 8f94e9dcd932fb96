// Host build of the library's FP32 solver arithmetic, for the CPU pins of
// the oracle's rounding-error bounds (tests/test_oracle_fp32_bounds.py).
// The solver header is written for host and device alike, with every
// operation explicitly rounded; built with -ffp-contract=off it gives, set
// for set, the bits the kernels give.  The inlier test is restated here in
// the kernels' order (threshold-folded form), since its device function uses
// device-only intrinsics.
#include <cmath>
#include <cstdint>

#include "../paper_2402_18008_gb300/csrc/aca_math.cuh"

static aca::Set set_of(const float *p)
{
    return aca::Set{p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7],
                    p[8], p[9], p[10], p[11], p[12], p[13], p[14], p[15]};
}

extern "C" void host_aca(const float *s, float *H, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        const aca::Set S = set_of(s + 16 * i);
        aca::AcaParts q;
        aca::aca_parts(S, q);
        aca::aca_compose(S, q, false, H + 9 * i);
    }
}

extern "C" void host_sks(const float *s, float *H, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) aca::sks_solve(set_of(s + 16 * i), H + 9 * i);
}

// The hypothesis of minimal set s as the RANSAC kernels form it (prescaled
// core, then scaled by a power of two so that its largest entry lies in
// [1, 2)) into H_out, and the test value e of every point: e < 0 <=> inlier.
extern "C" void host_test_e(const float *s, const float *corr, int64_t N, float thr, float *H_out, float *e_out)
{
    const aca::Set S = set_of(s);
    aca::AcaParts q;
    aca::aca_parts(S, q);
    float H[9];
    aca::aca_compose(S, q, true, H);
    const float sc = aca::pow2_inv_scale(aca::max_abs9(H));
    for (int i = 0; i < 9; ++i) H_out[i] = H[i] = H[i] * sc;
    float G[9];
    for (int i = 0; i < 6; ++i) G[i] = -H[i];
    G[6] = thr * H[6];
    G[7] = thr * H[7];
    G[8] = thr * H[8];
    const float rt = 1.0f / thr;
    for (int64_t i = 0; i < N; ++i) {
        const float *c = corr + 4 * i;
        const float Xs = c[2] * rt, Ys = c[3] * rt;
        const float w = std::fma(G[6], c[0], std::fma(G[7], c[1], G[8]));
        const float nu = std::fma(G[0], c[0], std::fma(G[1], c[1], G[2]));
        const float nv = std::fma(G[3], c[0], std::fma(G[4], c[1], G[5]));
        const float du = std::fma(Xs, w, nu), dv = std::fma(Ys, w, nv);
        e_out[i] = std::fma(du, du, std::fma(dv, dv, w * -w));
    }
}
