// ffb_fft.cuh -- in-register DFTs of one thread (lengths 2, 4, 8, 16, 32 and
// a real-input length 2, 4, 8, 16) and the constant twiddles they use; shared by the
// shared-memory grid kernel (ffb_grid.cu) and the ring FFT (ffb_ring.cu).
#pragma once
#include "ffb_internal.cuh"

// ---------------------------------------------------------------------------
// Register FFTs.  dft_reg<M>: a length-M DFT held in one thread's registers
// (M = 4, 8, 16: radix 4 with constant twiddles; M = 32: radix 2 over two
// length-16 DFTs).
// ---------------------------------------------------------------------------
template <int M>
__host__ __device__ constexpr int bitrev_c(int i) {
    int r = 0;
    for (int b = 1; b < M; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
    return r;
}

// W_16^e = exp(-2 pi i e / 16) for the e a radix-4 x 4 DFT needs
#define FFB_C1 0.92387953251128676f    // cos(pi/8)
#define FFB_S1 0.38268343236508977f    // sin(pi/8)
#define FFB_R2 0.70710678118654752f    // sqrt(1/2)
__device__ __forceinline__ float2 w16(int e) {
    switch (e & 15) {
        case 1: return make_float2(FFB_C1, -FFB_S1);
        case 2: return make_float2(FFB_R2, -FFB_R2);
        case 3: return make_float2(FFB_S1, -FFB_C1);
        case 4: return make_float2(0.f, -1.f);
        case 6: return make_float2(-FFB_R2, -FFB_R2);
        case 9: return make_float2(-FFB_C1, FFB_S1);
        default: return make_float2(1.f, 0.f);
    }
}

// cos / sin (2 pi e / 16), e = 0..15
__device__ __forceinline__ float cos16(int e) {
    constexpr float c[16] = {1.f, FFB_C1, FFB_R2, FFB_S1, 0.f, -FFB_S1, -FFB_R2, -FFB_C1,
                             -1.f, -FFB_C1, -FFB_R2, -FFB_S1, 0.f, FFB_S1, FFB_R2, FFB_C1};
    return c[e & 15];
}
__device__ __forceinline__ float sin16(int e) { return cos16(e + 12); }
// cos / sin (2 pi e / 32), e = 0..31
__device__ __forceinline__ float cos32(int e) {
    constexpr float c1 = 0.98078528040323044913f, c3 = 0.83146961230254523708f;
    constexpr float c5 = 0.55557023301960222474f, c7 = 0.19509032201612826785f;
    constexpr float c[32] = {1.f, c1, FFB_C1, c3, FFB_R2, c5, FFB_S1, c7, 0.f, -c7, -FFB_S1, -c5, -FFB_R2, -c3,
                             -FFB_C1, -c1, -1.f, -c1, -FFB_C1, -c3, -FFB_R2, -c5, -FFB_S1, -c7, 0.f, c7,
                             FFB_S1, c5, FFB_R2, c3, FFB_C1, c1};
    return c[e & 31];
}
__device__ __forceinline__ float sin32(int e) { return cos32(e + 24); }

// in-register length-M DFT, natural order in and out (forward)
template <int M>
__device__ __forceinline__ void dft_reg(float2 (&x)[M]) {
    if constexpr (M == 2) {
        const float2 a = x[0];
        x[0] = cadd(a, x[1]);
        x[1] = csub(a, x[1]);
    } else if constexpr (M == 4) {
        dft4<false>(x);
    } else if constexpr (M == 8) {
        float2 e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
        dft4<false>(e);
        dft4<false>(o);
        const float2 w[4] = {make_float2(1.f, 0.f), make_float2(FFB_R2, -FFB_R2), make_float2(0.f, -1.f),
                             make_float2(-FFB_R2, -FFB_R2)};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 t = (k == 0) ? o[0] : cmul(o[k], w[k]);
            x[k] = cadd(e[k], t);
            x[k + 4] = csub(e[k], t);
        }
    } else if constexpr (M == 32) {
        // radix 2 over two length-16 DFTs of the even and odd samples
        float2 e[16], o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            e[i] = x[2 * i];
            o[i] = x[2 * i + 1];
        }
        dft_reg<16>(e);
        dft_reg<16>(o);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            // W_32^k = (cos, -sin)(2 pi k / 32)
            const float2 t = (k == 0) ? o[0] : cmul(o[k], make_float2(cos32(k), -sin32(k)));
            x[k] = cadd(e[k], t);
            x[k + 16] = csub(e[k], t);
        }
    } else {
        static_assert(M == 16, "M in {2, 4, 8, 16, 32}");
        float2 y[4][4];   // y[n2][k1] = DFT4 over n1 of x[4 n1 + n2], times W16^{n2 k1}
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 v[4] = {x[n2], x[4 + n2], x[8 + n2], x[12 + n2]};
            dft4<false>(v);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = (n2 * k1 == 0) ? v[k1] : cmul(v[k1], w16(n2 * k1));
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 v[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
            dft4<false>(v);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = v[k2];
        }
    }
}

// length-H DFT of a real sequence u (H = 2, 4, 8), E[H - j] = conj E[j]
template <int H>
__device__ __forceinline__ void dft_real(const float (&u)[H], float2 (&E)[H]) {
    if constexpr (H == 2) {
        E[0] = make_float2(u[0] + u[1], 0.f);
        E[1] = make_float2(u[0] - u[1], 0.f);
    } else if constexpr (H == 4) {
        const float t0 = u[0] + u[2], t1 = u[0] - u[2], t2 = u[1] + u[3], t3 = u[1] - u[3];
        E[0] = make_float2(t0 + t2, 0.f);
        E[1] = make_float2(t1, -t3);
        E[2] = make_float2(t0 - t2, 0.f);
        E[3] = make_float2(t1, t3);
    } else if constexpr (H == 16) {
        // the complex length-16 DFT of the real sequence
#pragma unroll
        for (int i = 0; i < 16; ++i) E[i] = make_float2(u[i], 0.f);
        dft_reg<16>(E);
    } else {
        static_assert(H == 8, "H in {2, 4, 8, 16}");
        // even / odd samples: real length-4 DFTs A, B; E[j] = A[j] + W8^j B[j]
        const float a0 = u[0] + u[4], a1 = u[0] - u[4], a2 = u[2] + u[6], a3 = u[2] - u[6];
        const float b0 = u[1] + u[5], b1 = u[1] - u[5], b2 = u[3] + u[7], b3 = u[3] - u[7];
        const float A0 = a0 + a2, A2 = a0 - a2, B0 = b0 + b2, B2 = b0 - b2;
        const float2 A1 = make_float2(a1, -a3), B1 = make_float2(b1, -b3);
        const float2 wb = make_float2(FFB_R2 * (B1.x + B1.y), FFB_R2 * (B1.y - B1.x));   // W8 B1
        E[0] = make_float2(A0 + B0, 0.f);
        E[4] = make_float2(A0 - B0, 0.f);
        E[1] = cadd(A1, wb);
        E[5] = csub(A1, wb);
        E[2] = make_float2(A2, -B2);
        E[6] = make_float2(A2, B2);
        E[3] = cconj(E[5]);
        E[7] = cconj(E[1]);
    }
}

