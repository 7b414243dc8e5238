// Device FFT building blocks for the spectral Cahn-Hilliard passes.
//
// A CTA holds a tile of `npen` pencils of length L (complex float2) in shared
// memory; element i of pencil p lives at buf[i*es + p*ps]. A 1D transform
// along i is a sequence of Stockham (self-sorting) radix stages, one per
// factor of L (radices 16, 8, 4, 2, 5, 3). Stage s with radix R and
// Ns = product of earlier radices maps, for j in [0, L/R) with kk = j mod Ns,
//     v[t] = x[j + t L/R] * w_{Ns R}^{t kk}         (t < R)
//     y[(j - kk) R + kk + u Ns] = sum_t v[t] w_R^{t u} (u < R)
// which leaves the result in natural order after the last stage
// (Stockham autosort; Govindaraju et al., SC'08). Every stage is done in
// place: each thread loads its butterflies into registers, the CTA
// synchronises, then writes.
//
// Twiddles come from a table tw[m] = exp(-2 pi i m / L), m < L, computed on
// the host in FP64 and rounded to FP32; w_{Ns R}^{t kk} = tw[t kk L/(Ns R)].
// DIR = -1 is the forward transform (exp(-i..)), +1 the inverse, both
// unnormalised.
#pragma once
#include <cuda_runtime.h>

namespace evx {

constexpr int NT = 256;           // threads per CTA of every FFT pass
constexpr int TILE_CAP = 4096;    // max complex elements one fft_tile call transforms
constexpr int MAX_STAGES = 12;

struct Plan {
    int n;                 // number of stages
    int r[MAX_STAGES];     // radix of each stage
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (DIR=-1) or +i (DIR=+1)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}
// multiply by exp(DIR * i pi m / 8) for fixed m (constants of the 16th roots of unity)
template <int DIR, int m>
__device__ __forceinline__ float2 w16(float2 a) {
    constexpr float C1 = 0.92387953251128674f;  // cos(pi/8)
    constexpr float S1 = 0.38268343236508978f;  // sin(pi/8)
    constexpr float R2 = 0.70710678118654752f;  // cos(pi/4)
    constexpr int mm = m & 15;
    float c, s;  // exp(-i pi mm / 8) = c - i s  (forward); conj for inverse
    switch (mm) {
        case 0: return a;
        case 1: c = C1; s = S1; break;
        case 2: c = R2; s = R2; break;
        case 3: c = S1; s = C1; break;
        case 4: return mul_i<DIR>(a);
        case 5: c = -S1; s = C1; break;
        case 6: c = -R2; s = R2; break;
        case 7: c = -C1; s = S1; break;
        default: c = 1.f; s = 0.f; break;  // not used (m < 8 in radix-16)
    }
    // (a.x + i a.y)(c + i DIR s)
    const float ds = DIR < 0 ? -s : s;
    return make_float2(fmaf(a.x, c, -a.y * ds), fmaf(a.x, ds, a.y * c));
}

template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = mul_i<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// b + exp(DIR i pi m / 8) a for fixed m < 16, two FMAs per component for a general twiddle
template <int DIR, int m>
__device__ __forceinline__ float2 tw16_fma(float2 a, float2 b) {
    constexpr int mm = m & 7;
    constexpr float sg = (m & 8) ? -1.f : 1.f;  // w^(m + 8) = -w^m
    if (mm == 0) return sg > 0 ? cadd(b, a) : csub(b, a);
    if (mm == 4) return sg > 0 ? cadd(b, mul_i<DIR>(a)) : csub(b, mul_i<DIR>(a));
    constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508978f, R2 = 0.70710678118654752f;
    constexpr float c0 = mm == 1 ? C1 : mm == 2 ? R2 : mm == 3 ? S1 : mm == 5 ? -S1 : mm == 6 ? -R2 : -C1;
    constexpr float s0 = mm == 1 ? S1 : mm == 2 ? R2 : mm == 3 ? C1 : mm == 5 ? C1 : mm == 6 ? R2 : S1;
    constexpr float c = sg * c0;
    const float ds = DIR < 0 ? -sg * s0 : sg * s0;  // w = c + i ds
    return make_float2(fmaf(c, a.x, fmaf(-ds, a.y, b.x)), fmaf(c, a.y, fmaf(ds, a.x, b.y)));
}

// dft4 of (a0, w^m1 a1, w^m2 a2, w^m3 a3), w = exp(DIR i pi / 8): the twiddle
// products are taken into FMAs, and each difference of a butterfly is 2 x - (x + y)
template <int DIR, int m1, int m2, int m3>
__device__ __forceinline__ void dft4_tw(float2& a0, float2& a1, float2& a2, float2& a3) {
    constexpr bool triv2 = (m2 & 3) == 0;
    float2 t0, t1;
    if (triv2) {  // w^m2 in {1, DIR i, -1, -DIR i}
        const float2 r = (m2 & 4) ? mul_i<DIR>(a2) : a2;
        const float2 b2 = (m2 & 8) ? make_float2(-r.x, -r.y) : r;
        t0 = cadd(a0, b2);
        t1 = csub(a0, b2);
    } else {
        t0 = tw16_fma<DIR, m2>(a2, a0);
        t1 = make_float2(fmaf(2.f, a0.x, -t0.x), fmaf(2.f, a0.y, -t0.y));
    }
    const float2 u1 = w16<DIR, m1>(a1);
    const float2 t2 = tw16_fma<DIR, m3>(a3, u1);
    const float2 t3 = mul_i<DIR>(make_float2(fmaf(2.f, u1.x, -t2.x), fmaf(2.f, u1.y, -t2.y)));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2* v) { dft2<DIR>(v[0], v[1]); }
};
template <int DIR>
struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2* v) { dft4<DIR>(v[0], v[1], v[2], v[3]); }
};
template <int DIR>
struct Dft<8, DIR> {
    // decimation in time: E = DFT4(even), O = DFT4(odd), X_k = E_k + w8^k O_k
    __device__ __forceinline__ static void run(float2* v) {
        float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<DIR>(e0, e1, e2, e3);
        dft4<DIR>(o0, o1, o2, o3);
        o1 = w16<DIR, 2>(o1);
        o2 = w16<DIR, 4>(o2);
        o3 = w16<DIR, 6>(o3);
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    }
};
template <int DIR>
struct Dft<16, DIR> {
    // 4 x 4: E_{n2}[k1] = DFT4_{n1}(a[4 n1 + n2]); twiddle w16^{n2 k1};
    // X[k1 + 4 k2] = DFT4_{n2}(...)[k2]
    __device__ __forceinline__ static void run(float2* v) {
        dft4<DIR>(v[0], v[4], v[8], v[12]);
        dft4<DIR>(v[1], v[5], v[9], v[13]);
        dft4<DIR>(v[2], v[6], v[10], v[14]);
        dft4<DIR>(v[3], v[7], v[11], v[15]);
        // after dft4 on (v[n2], v[4+n2], v[8+n2], v[12+n2]) slot 4*k1 + n2 holds E_{n2}[k1];
        // row k1 is twiddled by w16^(k1 n2) and transformed along n2
        dft4<DIR>(v[0], v[1], v[2], v[3]);
        dft4_tw<DIR, 1, 2, 3>(v[4], v[5], v[6], v[7]);
        dft4_tw<DIR, 2, 4, 6>(v[8], v[9], v[10], v[11]);
        dft4_tw<DIR, 3, 6, 9>(v[12], v[13], v[14], v[15]);
        // slot 4*k1 + k2 now holds X[k1 + 4 k2]; transpose to natural order
        float2 t;
        t = v[1]; v[1] = v[4]; v[4] = t;
        t = v[2]; v[2] = v[8]; v[8] = t;
        t = v[3]; v[3] = v[12]; v[12] = t;
        t = v[6]; v[6] = v[9]; v[9] = t;
        t = v[7]; v[7] = v[13]; v[13] = t;
        t = v[11]; v[11] = v[14]; v[14] = t;
    }
};
// multiply by exp(DIR * i pi m / 16) for fixed m < 16 (32nd roots of unity)
template <int DIR, int m>
__device__ __forceinline__ float2 w32(float2 a) {
    // cos(pi j / 16), j = 0..8
    constexpr float C[9] = {1.0f,
                            0.98078528040323043f,
                            0.92387953251128674f,
                            0.83146961230254524f,
                            0.70710678118654752f,
                            0.55557023301960218f,
                            0.38268343236508978f,
                            0.19509032201612825f,
                            0.0f};
    if (m == 0) return a;
    if (m == 8) return mul_i<DIR>(a);
    // exp(-i pi m/16) = cos - i sin; for m > 8: cos(pi m/16) = -cos(pi (16-m)/16)
    constexpr float c = m <= 8 ? C[m] : -C[16 - m];
    constexpr float s = m <= 8 ? C[8 - m] : C[m - 8];
    const float ds = DIR < 0 ? -s : s;
    return make_float2(fmaf(a.x, c, -a.y * ds), fmaf(a.x, ds, a.y * c));
}

template <int DIR>
struct Dft<32, DIR> {
    // decimation in time: E = DFT16(even), O = DFT16(odd), X_k = E_k + w32^k O_k,
    // X_{k+16} = E_k - w32^k O_k. For a general twiddle the sum takes the product
    // into two FMAs per component and the difference is 2 E_k - X_k (one FMA per
    // component): 6 instructions per butterfly instead of 8.
    template <int k>
    __device__ __forceinline__ static void comb(float2* v, float2* e, float2* o) {
        if (k == 0 || k == 8) {
            const float2 t = w32<DIR, k>(o[k]);
            v[k] = cadd(e[k], t);
            v[k + 16] = csub(e[k], t);
            return;
        }
        constexpr float C[9] = {1.0f,
                                0.98078528040323043f,
                                0.92387953251128674f,
                                0.83146961230254524f,
                                0.70710678118654752f,
                                0.55557023301960218f,
                                0.38268343236508978f,
                                0.19509032201612825f,
                                0.0f};
        constexpr float c = k <= 8 ? C[k] : -C[16 - k];
        constexpr float sn = k <= 8 ? C[8 - k] : C[k - 8];
        const float ds = DIR < 0 ? -sn : sn;  // w32^k = c + i ds
        const float2 ek = e[k], ok = o[k];
        const float2 s = make_float2(fmaf(c, ok.x, fmaf(-ds, ok.y, ek.x)), fmaf(c, ok.y, fmaf(ds, ok.x, ek.y)));
        v[k] = s;
        v[k + 16] = make_float2(fmaf(2.f, ek.x, -s.x), fmaf(2.f, ek.y, -s.y));
    }
    __device__ __forceinline__ static void run(float2* v) {
        float2 e[16], o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        Dft<16, DIR>::run(e);
        Dft<16, DIR>::run(o);
        comb<0>(v, e, o);  comb<1>(v, e, o);  comb<2>(v, e, o);  comb<3>(v, e, o);
        comb<4>(v, e, o);  comb<5>(v, e, o);  comb<6>(v, e, o);  comb<7>(v, e, o);
        comb<8>(v, e, o);  comb<9>(v, e, o);  comb<10>(v, e, o); comb<11>(v, e, o);
        comb<12>(v, e, o); comb<13>(v, e, o); comb<14>(v, e, o); comb<15>(v, e, o);
    }
};
template <int DIR>
struct Dft<1, DIR> {
    __device__ __forceinline__ static void run(float2*) {}
};

template <int DIR>
struct Dft<3, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        constexpr float H3 = 0.86602540378443865f;  // sin(2 pi / 3)
        float2 t = cadd(v[1], v[2]);
        float2 s = csub(v[1], v[2]);
        float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        float2 r = mul_i<DIR>(cscale(s, H3));  // DIR i sin(2pi/3) s
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
};
template <int DIR>
struct Dft<5, DIR> {
    __device__ __forceinline__ static void run(float2* v) {
        constexpr float C1 = 0.30901699437494742f;   // cos(2 pi/5)
        constexpr float C2 = -0.80901699437494742f;  // cos(4 pi/5)
        constexpr float S1 = 0.95105651629515357f;   // sin(2 pi/5)
        constexpr float S2 = 0.58778525229247313f;   // sin(4 pi/5)
        float2 t1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
        float2 t2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
        float2 a0 = v[0];
        float2 m1 = make_float2(a0.x + C1 * t1.x + C2 * t2.x, a0.y + C1 * t1.y + C2 * t2.y);
        float2 m2 = make_float2(a0.x + C2 * t1.x + C1 * t2.x, a0.y + C2 * t1.y + C1 * t2.y);
        // forward: X1 = m1 - i(S1 d1 + S2 d2), X2 = m2 - i(S2 d1 - S1 d2)
        float2 q1 = mul_i<DIR>(make_float2(S1 * d1.x + S2 * d2.x, S1 * d1.y + S2 * d2.y));
        float2 q2 = mul_i<DIR>(make_float2(S2 * d1.x - S1 * d2.x, S2 * d1.y - S1 * d2.y));
        v[0] = make_float2(a0.x + t1.x + t2.x, a0.y + t1.y + t2.y);
        v[1] = cadd(m1, q1);
        v[4] = csub(m1, q1);
        v[2] = cadd(m2, q2);
        v[3] = csub(m2, q2);
    }
};

// multiply by exp(DIR * 2 pi i m / 20) for fixed m (20th roots of unity)
template <int DIR, int m>
__device__ __forceinline__ float2 w20(float2 a) {
    // cos(pi j / 10), j = 0..5
    constexpr float C[6] = {1.0f, 0.95105651629515357f, 0.80901699437494742f, 0.58778525229247313f,
                            0.30901699437494742f, 0.0f};
    constexpr int mm = m % 20;
    if (mm == 0) return a;
    if (mm == 5) return mul_i<DIR>(a);
    if (mm == 10) return make_float2(-a.x, -a.y);
    if (mm == 15) return mul_i<-DIR>(a);
    // cos and sin of pi mm / 10 from the first quadrant by symmetry
    constexpr int q = mm % 10, qq = q <= 5 ? q : 10 - q;
    constexpr float cq = q <= 5 ? C[qq] : -C[qq];  // cos(pi q / 10)
    constexpr float sq = C[5 - qq];                // sin(pi q / 10) >= 0
    constexpr float c = mm < 10 ? cq : -cq, s = mm < 10 ? sq : -sq;
    const float ds = DIR < 0 ? -s : s;
    return make_float2(fmaf(a.x, c, -a.y * ds), fmaf(a.x, ds, a.y * c));
}

// length 10 = 2 x 5, decimation in time: F_r = DFT5(x[2 m + r]),
// X[k + 5 q] = F_0[k] + (-1)^q w_10^k F_1[k]
template <int DIR>
struct Dft<10, DIR> {
    template <int k>
    __device__ __forceinline__ static void comb(float2* v, const float2* e, const float2* o) {
        const float2 t = w20<DIR, 2 * k>(o[k]);
        v[k] = cadd(e[k], t);
        v[k + 5] = csub(e[k], t);
    }
    __device__ __forceinline__ static void run(float2* v) {
        float2 e[5], o[5];
#pragma unroll
        for (int m = 0; m < 5; ++m) {
            e[m] = v[2 * m];
            o[m] = v[2 * m + 1];
        }
        Dft<5, DIR>::run(e);
        Dft<5, DIR>::run(o);
        comb<0>(v, e, o); comb<1>(v, e, o); comb<2>(v, e, o); comb<3>(v, e, o); comb<4>(v, e, o);
    }
};

// length 20 = 4 x 5, decimation in time: F_r = DFT5(x[4 m + r]) (r < 4),
// X[k + 5 q] = DFT4_r(w_20^{r k} F_r[k])[q]
template <int DIR>
struct Dft<20, DIR> {
    template <int k>
    __device__ __forceinline__ static void comb(float2* v, float2 (&f)[4][5]) {
        float2 g0 = f[0][k], g1 = w20<DIR, k>(f[1][k]), g2 = w20<DIR, 2 * k>(f[2][k]), g3 = w20<DIR, 3 * k>(f[3][k]);
        dft4<DIR>(g0, g1, g2, g3);
        v[k] = g0;
        v[k + 5] = g1;
        v[k + 10] = g2;
        v[k + 15] = g3;
    }
    __device__ __forceinline__ static void run(float2* v) {
        float2 f[4][5];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int m = 0; m < 5; ++m) f[r][m] = v[4 * m + r];
            Dft<5, DIR>::run(f[r]);
        }
        comb<0>(v, f); comb<1>(v, f); comb<2>(v, f); comb<3>(v, f); comb<4>(v, f);
    }
};

// Tile descriptor: pencil p, element i at buf[i*es + p*ps].
struct Tile {
    float2* buf;
    int L;
    int npen;
    int es;
    int ps;
};

// One in-place Stockham stage of radix R. PEN_FAST: consecutive threads take
// consecutive pencils (tiles whose pencils are adjacent in memory); otherwise
// consecutive butterflies of one pencil.
template <int R, int DIR, bool PEN_FAST>
__device__ __forceinline__ void fft_stage(const Tile& t, int Ns, const float2* __restrict__ tw) {
    constexpr int KMAX = (TILE_CAP + R * NT - 1) / (R * NT);
    const int LR = t.L / R;
    const int nb = LR * t.npen;
    const int tws = t.L / (Ns * R);
    float2 v[KMAX][R];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int b = threadIdx.x + k * NT;
        if (b < nb) {
            int p, j;
            if (PEN_FAST) { p = b % t.npen; j = b / t.npen; }
            else          { j = b % LR;     p = b / LR; }
            const int kk = j % Ns;
            const float2* src = t.buf + p * t.ps + j * t.es;
#pragma unroll
            for (int r = 0; r < R; ++r) v[k][r] = src[r * LR * t.es];
            if (Ns > 1) {
                const int step = tws * kk;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw[r * step];
                    if (DIR > 0) w.y = -w.y;
                    v[k][r] = cmul(v[k][r], w);
                }
            }
            Dft<R, DIR>::run(v[k]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int b = threadIdx.x + k * NT;
        if (b < nb) {
            int p, j;
            if (PEN_FAST) { p = b % t.npen; j = b / t.npen; }
            else          { j = b % LR;     p = b / LR; }
            const int kk = j % Ns;
            float2* dst = t.buf + p * t.ps + ((j - kk) * R + kk) * t.es;
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r * Ns * t.es] = v[k][r];
        }
    }
    __syncthreads();
}

// Full 1D transform of every pencil of the tile (caller has synchronised;
// L * npen <= TILE_CAP). Not inlined: one copy serves every kernel.
template <int DIR, bool PEN_FAST>
__device__ __noinline__ void fft_tile(const Tile& t, const Plan& pl, const float2* __restrict__ tw) {
    int Ns = 1;
    for (int s = 0; s < pl.n; ++s) {
        const int R = pl.r[s];
        switch (R) {
            case 16: fft_stage<16, DIR, PEN_FAST>(t, Ns, tw); break;
            case 8:  fft_stage<8, DIR, PEN_FAST>(t, Ns, tw); break;
            case 4:  fft_stage<4, DIR, PEN_FAST>(t, Ns, tw); break;
            case 2:  fft_stage<2, DIR, PEN_FAST>(t, Ns, tw); break;
            case 5:  fft_stage<5, DIR, PEN_FAST>(t, Ns, tw); break;
            case 3:  fft_stage<3, DIR, PEN_FAST>(t, Ns, tw); break;
            default: break;
        }
        Ns *= R;
    }
}

}  // namespace evx
