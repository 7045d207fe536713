// thermo.cu -- partition function and moments from the degeneracy table (arXiv:1110.2561,
// Eq. 2 summed over the table g(E, M) of Sec. 2), on a grid of temperatures T and fields h.
//
// Z(T, h) = sum_{E,M} g(E, M) exp(-(E - h M) / T) factors exactly over M:
//   Z = sum_M exp(h M / T) A_T(M),   A_T(M) = sum_E g(E, M) exp(-E / T).
// Stage 1 (per T and M, independent of h) keeps, log-shifted by the largest term,
// L_T(M) = ln A_T(M) and the conditional mean and variance of E at fixed M. Stage 2 (per T and
// h) combines them over the N + 1 values of M with a log-sum-exp, in one pass:
//   <H> = sum_M p(M) (mu_E(M) - h M),  Var(H) = sum_M p(M) [var_E(M) + (mu_E(M) - h M - <H>)^2],
// with p(M) proportional to exp(L_T(M) + h M / T). The squares are taken about the dominant
// column M* (the mode of p) and the mean correction subtracted at the end; the mean lies within a
// few standard deviations of the mode, so C = Var(H)/T^2 and chi = Var(M)/T lose at most a small
// factor to cancellation.
//
// The magnetisation statistics <|M|>, <M^2>, <M^4> and Binder's cumulant 1 - <M^4>/(3<M^2>^2)
// depend on (T, h) only through p(M), so they come from the same stage-2 weights. Passes whose
// outputs were not requested are skipped (the E-variance pass of stage 1 when C is not asked for,
// the variance pass of stage 2 when neither C nor chi is).
//
// FP64: everything in double. FP32: the counts are converted to ln g in double once and rounded
// to float; every exponential and every sum runs in float, relative to the column maximum in
// stage 1 and to the dominant column of each (T, h) point in stage 2, whose large offsets are
// carried as pairs of floats; ln Z is finished in double from the float sum.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "isg_internal.h"
#include "nvtx_range.h"

namespace isg {

DeviceInfo device_info();

constexpr int kInlineGrid = 1024;   // T and h values passed inside the kernel parameters
constexpr int kThermoOuts = 9;      // logZ, E, M, C, chi, absM, M2, M4, binder

struct ThermoArgs {
    const int64_t* g;   // n_e x n_m counts
    const double* T;    // nT (device), or NULL: inline[0 .. nT)
    const double* h;    // nh (device), or NULL: inline[nT .. nT + nh)
    double* logZ;
    double* E;
    double* M;
    double* C;
    double* chi;
    double* absM;       // <|M|>
    double* M2;         // <M^2>
    double* M4;         // <M^4>
    double* binder;     // 1 - <M^4> / (3 <M^2>^2)
    int n, n_e, n_m, nT, nh;
    int64_t e_min;
    int e0, eg, n_on;   // energy sublattice of the graph: public bins e0 + eg k, k < n_on
    int cluster;        // CTAs per temperature (a thread-block cluster when > 1)
};

// Kernel parameters: the arguments plus small grids inline, so a call on a small grid needs no
// host-to-device copy.
struct ThermoParams {
    ThermoArgs a;
    double grid[kInlineGrid];
};

template <class F> __device__ __forceinline__ F ex(F x);
template <> __device__ __forceinline__ double ex<double>(double x) { return exp(x); }
template <> __device__ __forceinline__ float ex<float>(float x) { return expf(x); }
template <class F> __device__ __forceinline__ F lg(F x);
template <> __device__ __forceinline__ double lg<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float lg<float>(float x) { return logf(x); }

// Fused multiply-add, absolute value and maximum in the working precision. The float versions
// are named explicitly so that no argument is promoted to double (double arithmetic runs on
// this GPU's narrow FP64 pipe).
__device__ __forceinline__ float fmaF(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaF(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float absF(float x) { return fabsf(x); }
__device__ __forceinline__ double absF(double x) { return fabs(x); }
__device__ __forceinline__ float maxF(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double maxF(double a, double b) { return fmax(a, b); }

// -inf marks empty bins and columns. For double the test reads the high word on the integer
// pipe instead of occupying the narrow FP64 pipe; it is exact here because no finite double has an
// all-ones exponent (and no value here is a NaN).
__device__ __forceinline__ bool is_neg_inf(double x) { return __double2hiint(x) == (int)0xfff00000; }
__device__ __forceinline__ bool is_neg_inf(float x) { return x == -INFINITY; }

template <class F>
__device__ __forceinline__ F warp_max(F v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = maxF(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <class F>
__device__ __forceinline__ F warp_sum(F v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of two values with five additions per lane instead of ten: at the first level each
// half-warp keeps one value and adds its partner's copy of it. Returns the sum of a in lanes
// 0..15 and of b in lanes 16..31.
template <class F>
__device__ __forceinline__ F warp_sum2(F a, F b) {
    const bool hi = threadIdx.x & 16;
    F v = (hi ? b : a) + __shfl_xor_sync(0xffffffffu, hi ? a : b, 16);
#pragma unroll
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of eight values with nine additions per lane instead of forty (the same halving at
// the first three levels). On return v[j] holds the full sum of value j in every lane.
template <class F>
__device__ __forceinline__ void warp_sum8(F (&v)[8]) {
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    F w[4], x[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = (b4 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[i + 4], 16);
#pragma unroll
    for (int i = 0; i < 2; ++i) x[i] = (b3 ? w[i + 2] : w[i]) + __shfl_xor_sync(0xffffffffu, b3 ? w[i] : w[i + 2], 8);
    F y = (b2 ? x[1] : x[0]) + __shfl_xor_sync(0xffffffffu, b2 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(0xffffffffu, y, 2);
    y += __shfl_xor_sync(0xffffffffu, y, 1);
    // lane bits (4, 3, 2) name the value whose sum the lane now holds
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __shfl_sync(0xffffffffu, y, ((j & 4) << 2) | ((j & 2) << 2) | ((j & 1) << 2));
}

// ln g for every bin, computed in double from the int64 count and stored in double and (rounded)
// in float; -inf marks an empty bin.
__global__ void log_counts_kernel(const int64_t* g, int nbins, double* lng, float* lngf, float* lnglo) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbins; i += gridDim.x * blockDim.x) {
        const int64_t c = g[i];
        const double l = c > 0 ? log((double)c) : -INFINITY;
        lng[i] = l;
        lngf[i] = (float)l;
        lnglo[i] = c > 0 ? (float)(l - (double)(float)l) : 0.0f;     // remainder: lngf + lnglo = ln g
    }
}

// One pass over every bin of a column for stage 1 (lane-strided, public bins e of column m in
// table tab, energies El + Es j in precision U): the reference bin, the one maximising
// ln g - E/T, and whether any count lies off the graph's energy sublattice (bins e0 + eg k,
// e <= e_last; r is (e - e0) mod eg for the lane's first bin, stepped by r32 = 32 mod eg).
// Returns the ballot of the lanes holding the warp maximum (0: empty column); the lane's best
// bin goes to ebest and its off-sublattice finding to off.
template <class U>
__device__ __forceinline__ unsigned column_scan(const U* tab, int n_m, int m, int n_e, int e0, int eg, int e_last, int r,
                                                int r32, U El, U Es, U invT, int& ebest, bool& off) {
    U xmax = (U)-INFINITY;
    ebest = 0;
    off = false;
    U En = El;
    for (int e = threadIdx.x & 31; e < n_e; e += 32, En += Es) {
        const U l = tab[(size_t)e * n_m + m];
        const bool on = r == 0 && e >= e0 && e <= e_last;
        r += r32;
        if (r >= eg) r -= eg;
        if (is_neg_inf(l)) continue;
        if (!on) off = true;
        const U x = fmaF(-En, invT, l);
        if (x > xmax) { xmax = x; ebest = e; }
    }
    const U wmax = warp_max(xmax);
    return __ballot_sync(0xffffffffu, xmax == wmax && wmax != (U)-INFINITY);
}

// Dominant column of a stage-2 point: over m = mfirst, mfirst + mstep, ..., the one maximising
// Lr[m] + (h/T) M_m, searched in precision U (Lr in that precision).
template <class U>
__device__ __forceinline__ int dominant_column(const U* Lr, int n, int n_m, int mfirst, int mstep, U hT, bool by_warp) {
    U amax = (U)-INFINITY;
    int ms = 0;
    U Mm = (U)(2 * mfirst - n);
    const U Ms = (U)(2 * mstep);
    for (int m = mfirst; m < n_m; m += mstep, Mm += Ms) {
        const U lr = Lr[m];
        if (is_neg_inf(lr)) continue;
        const U am = fmaF(hT, Mm, lr);
        if (am > amax) { amax = am; ms = m; }
    }
    if (by_warp) {                        // the lowest lane holding the warp maximum names m*
        const U wm = warp_max(amax);
        const unsigned hit = __ballot_sync(0xffffffffu, amax == wm && wm != (U)-INFINITY);
        ms = __shfl_sync(0xffffffffu, ms, hit ? __ffs(hit) - 1 : 0);
    }
    return ms;
}

template <class F> __device__ __forceinline__ const F* pick(const double* d, const float* f);
template <> __device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <> __device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

// One CTA per temperature, or, for grids of fewer temperatures than half the SMs, one cluster of
// a.cluster CTAs per temperature: the cluster's CTAs share stage 1's columns and write their
// results into the shared memory of the cluster's first CTA, which alone runs the rest.
// Shared memory: L[n_m] (double), mu, var, Lr, Llo, cs0, qin [n_m] (F), ces[n_m] (int), Lrf[n_m]
// (float).
//
// Stage 1 walks, per column, the public energy bins e0 + eg k (k < n_on) on which the graph's
// energies E = e_lo + G k' lie (eg = G / 2: every other bin on lattices with an energy stride of
// 4); a column that holds counts off those bins (a table that is not this graph's) is walked
// bin by bin.
//
// Stage 2 forms every exponent relative to the dominant column m* of its (T, h) point:
//   d_m = (Lr[m] - Lr[m*]) + (Llo[m] - Llo[m*]) + (h/T)(M_m - M_m*),
// with Lr + Llo = L - max L and h/T = hT + hTlo held as pairs of the working precision (for
// float this is what keeps ln Z accurate to ~1e-7 although L - max L reaches hundreds), and
// finishes ln Z = max L + (L[m*] - max L) + (h/T) M_m* + ln(sum exp d_m) in double.
//
// The reference bin of a column and the dominant column of a point are searched in float in
// both precisions: they only need to lie near the maximum (every weight is formed relative to
// them, and a reference a rounding error below the maximum leaves the weights near 1).
template <class F>
__global__ void __launch_bounds__(1024) thermo_kernel(const __grid_constant__ ThermoParams P, const double* lngd,
                                                     const float* lngf, const float* lnglo) {
    namespace cg = cooperative_groups;
    const ThermoArgs& a = P.a;
    const double* Tv = a.T ? a.T : P.grid;
    const double* hv = a.h ? a.h : P.grid + a.nT;
    const F* lng = pick<F>(lngd, lngf);
    constexpr bool pair = sizeof(F) == sizeof(float);   // float: ln g carried as lngf + lnglo
    extern __shared__ __align__(16) unsigned char sm[];
    double* L = reinterpret_cast<double*>(sm);
    F* mu = reinterpret_cast<F*>(L + a.n_m);
    F* var = mu + a.n_m;
    F* Lr = var + a.n_m;                 // L - max L, rounded to F (-inf: empty column)
    F* Llo = Lr + a.n_m;                 // the rounding remainder of Lr
    F* cs0 = Llo + a.n_m;                // per column: sum of weights relative to the largest
    // FP64, one thread per point: qin[m] = exp(Lr[m] - Lr[m-1]), the h-independent factor between
    // neighbouring columns' weights (0 for m = 0 or an empty neighbour)
    F* qin = cs0 + a.n_m;
    int* ces = reinterpret_cast<int*>(qin + a.n_m);   // per column: the largest bin e* (-1: empty)
    float* Lrf = reinterpret_cast<float*>(ces + a.n_m);
    __shared__ double s_Lmax;
    const int csz = a.cluster;
    const int rank = csz > 1 ? (int)cg::this_cluster().block_rank() : 0;
    const int it = blockIdx.x / csz;
    const double T = Tv[it], invTd = 1.0 / T;
    const F invT = (F)invTd, invTlo = (F)(invTd - (double)invT), invT2 = (F)(invTd * invTd);
    const float invTf = (float)invTd;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    // stage-1 results go to the cluster's first CTA (distributed shared memory); every CTA of
    // the cluster must be running before any writes into another's shared memory
    F *mu_d = mu, *var_d = var, *cs0_d = cs0;
    int* ces_d = ces;
    if (csz > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        mu_d = cl.map_shared_rank(mu, 0);
        var_d = cl.map_shared_rank(var, 0);
        cs0_d = cl.map_shared_rank(cs0, 0);
        ces_d = cl.map_shared_rank(ces, 0);
    }

    // Stage 1: per column M (one warp each).
    // Energies E_e = e_min + 2e are exact in float (|E| < 2^24); the loops step them in float
    // instead of converting e, since integer-to-float conversions share the slow FP64 pipe on
    // this GPU. Lane energies of the sublattice walk (S) and of the dense walk (D):
    const float ElS = (float)(a.e_min + 2 * (a.e0 + a.eg * lane)), EsS = (float)(64 * a.eg);
    const float ElD = (float)(a.e_min + 2 * lane), EsD = 64.0f;
    const bool sparse_graph = a.eg > 1 || a.n_on < a.n_e;
    // The reference search runs in float where float keeps it within ~1e-3 of the maximum:
    // every compared value is below S/T + 45 in magnitude, so for S/T <= 1e4 its rounding error
    // stays below 1e-3. Otherwise (FP64 only) it runs in double.
    const bool search_float = pair || (double)(-a.e_min) * invTd <= 1e4;
    const double ElDd = (double)ElD, EsDd = 64.0;
    const int e_last = a.e0 + a.eg * (a.n_on - 1), r32 = 32 % a.eg;
    const int r0 = ((lane - a.e0) % a.eg + a.eg) % a.eg;
    for (int m = rank + csz * warp; m < a.n_m; m += csz * nw) {
        int ebest;
        bool off;
        // a lane holding the maximum names the reference energy (any tie is fine)
        const unsigned hit =
            search_float ? column_scan<float>(lngf, a.n_m, m, a.n_e, a.e0, a.eg, e_last, r0, r32, ElD, EsD, invTf, ebest, off)
                         : column_scan<double>(lngd, a.n_m, m, a.n_e, a.e0, a.eg, e_last, r0, r32, ElDd, EsDd, invTd, ebest,
                                               off);
        if (!hit) {
            if (lane == 0) { ces_d[m] = -1; mu_d[m] = 0; var_d[m] = 0; }
            continue;
        }
        const int es = __shfl_sync(0xffffffffu, ebest, __ffs(hit) - 1);
        // the exponential passes walk the sublattice unless the column holds counts off it
        const bool dense = !sparse_graph || __any_sync(0xffffffffu, off);
        const int cb = dense ? 0 : a.e0, cs = dense ? 1 : a.eg, cn = dense ? a.n_e : a.n_on;
        const float El = dense ? ElD : ElS, Es = dense ? EsD : EsS;
        // exponents relative to the reference bin e*: (ln g_e - ln g_e*) - (E_e - E_e*) / T, the
        // differences formed from the (hi, lo) pairs so no large value is rounded on the way
        const size_t is = (size_t)es * a.n_m + m;
        const F ls = lng[is];
        F lls = 0;
        if constexpr (pair) lls = (F)lnglo[is];
        const F Eref = (F)(a.e_min + 2 * es);
        const F ElF = (F)El, EsF = (F)Es;
        auto arg = [&](int e, F l, F dE) -> F {
            if constexpr (pair) {
                const F dl = (l - ls) + ((F)lnglo[(size_t)e * a.n_m + m] - lls);
                return dl - fmaF(dE, invT, dE * invTlo);
            } else {
                return fmaF(-dE, invT, l - ls);
            }
        };
        // weights of the first kCache bins of each lane stay in registers for the second pass
        constexpr int kCache = 8;
        F wc[kCache];
        F s0 = 0, s1 = 0;
#pragma unroll
        for (int j = 0; j < kCache; ++j) {
            const int k = lane + 32 * j;
            wc[j] = 0;
            if (k >= cn) continue;
            const int e = cb + cs * k;
            const F l = lng[(size_t)e * a.n_m + m];
            if (is_neg_inf(l)) continue;
            const F dE = fmaF(EsF, (F)j, ElF) - Eref;
            const F w = ex<F>(arg(e, l, dE));
            wc[j] = w;
            s0 += w;
            s1 += w * dE;
        }
        {
            F En = fmaF(EsF, (F)kCache, ElF);
            for (int k = lane + 32 * kCache; k < cn; k += 32, En += EsF) {
                const int e = cb + cs * k;
                const F l = lng[(size_t)e * a.n_m + m];
                if (is_neg_inf(l)) continue;
                const F dE = En - Eref;
                const F w = ex<F>(arg(e, l, dE));
                s0 += w;
                s1 += w * dE;
            }
        }
        {
            const F v = warp_sum2(s0, s1);
            s0 = __shfl_sync(0xffffffffu, v, 0);
            s1 = __shfl_sync(0xffffffffu, v, 16);
        }
        const F inv0 = (F)1 / s0;
        const F m1 = Eref + s1 * inv0;
        F s2 = 0;
        if (a.C) {
#pragma unroll
            for (int j = 0; j < kCache; ++j) {
                const F d = fmaF(EsF, (F)j, ElF) - m1;
                s2 += wc[j] * d * d;
            }
            F En = fmaF(EsF, (F)kCache, ElF);
            for (int k = lane + 32 * kCache; k < cn; k += 32, En += EsF) {
                const int e = cb + cs * k;
                const F l = lng[(size_t)e * a.n_m + m];
                if (is_neg_inf(l)) continue;
                const F w = ex<F>(arg(e, l, En - Eref));
                const F d = En - m1;
                s2 += w * d * d;
            }
            s2 = warp_sum(s2);
        }
        if (lane == 0) {
            cs0_d[m] = s0;
            ces_d[m] = es;
            mu_d[m] = m1;
            var_d[m] = s2 * inv0;
        }
    }
    if (csz > 1) {
        cg::this_cluster().sync();           // release / acquire: the first CTA sees every column
        if (rank != 0) return;
    } else {
        __syncthreads();
    }
    // L_T(M) in double, the columns side by side (double arithmetic occupies the narrow FP64 pipe
    // for a whole warp even with one lane active); ln of the relative sum s0 in [1, n_e] is taken
    // in the working precision.
    for (int m = threadIdx.x; m < a.n_m; m += blockDim.x) {
        const int es = ces[m];
        L[m] = es < 0 ? -INFINITY
                      : (lngd[(size_t)es * a.n_m + m] - (double)(a.e_min + 2 * es) * invTd) + (double)lg<F>(cs0[m]);
    }
    __syncthreads();
    if (warp == 0) {
        double mx = -INFINITY;
        for (int m = lane; m < a.n_m; m += 32) mx = fmax(mx, L[m]);
        mx = warp_max(mx);
        if (lane == 0) s_Lmax = mx;
    }
    __syncthreads();
    const double Lmax = s_Lmax;
    for (int m = threadIdx.x; m < a.n_m; m += blockDim.x) {
        if (L[m] == -INFINITY) { Lr[m] = (F)-INFINITY; Llo[m] = 0; Lrf[m] = -INFINITY; continue; }
        const double r = L[m] - Lmax;
        Lr[m] = (F)r;
        Llo[m] = (F)(r - (double)(F)r);
        Lrf[m] = (float)r;
    }
    const bool by_warp = a.nh < 64;
    constexpr bool kChain = sizeof(F) == sizeof(double);
    if (kChain && !by_warp) {
        __syncthreads();
        for (int m = threadIdx.x; m < a.n_m; m += blockDim.x)
            qin[m] = (m == 0 || L[m] == -INFINITY || L[m - 1] == -INFINITY) ? (F)0 : ex<F>(Lr[m] - Lr[m - 1]);
    }
    __syncthreads();

    // Stage 2. Many field values: one thread per point, a serial loop over M. Few field values
    // (fewer than 64): one warp per point, lanes over M, shuffle reductions.
    const bool mag = a.absM || a.M2 || a.M4 || a.binder, variances = a.C || a.chi;
    const int step = by_warp ? nw : blockDim.x, first = by_warp ? warp : threadIdx.x;
    const int mstep = by_warp ? 32 : 1, mfirst = by_warp ? lane : 0;
    // M_m - M_m* stepped in F as well: 2 * mstep per iteration.
    const F dstep = (F)(2 * mstep);
    for (int ih = first; ih < a.nh; ih += step) {
        const double hd = hv[ih], hTd = hd * invTd;
        const F hT = (F)hTd, hTlo = (F)(hTd - (double)hT), hF = (F)hd;
        // In float where float keeps the choice within ~1e-3 of the maximum: the contenders' Lr
        // lie within 2 |h/T| N of 0, so for |h/T| N <= 5e3 every compared value is below 1.5e4.
        int ms;
        if constexpr (pair) ms = dominant_column<float>(Lr, a.n, a.n_m, mfirst, mstep, hT, by_warp);
        else
            ms = fabs(hTd) * a.n <= 5e3 ? dominant_column<float>(Lrf, a.n, a.n_m, mfirst, mstep, (float)hTd, by_warp)
                                        : dominant_column<double>(Lr, a.n, a.n_m, mfirst, mstep, hTd, by_warp);
        // One pass: weights p_m and the moments of dM = M_m - M_m* and dH = H_m - H_m* about the
        // dominant column. m* is the mode of p, so the mean lies within a few standard deviations
        // of it and Var = <d^2> - <d>^2 loses at most a small factor to cancellation.
        const F Ls = Lr[ms], Lls = Llo[ms], mus = mu[ms];
        const int Ms = 2 * ms - a.n;
        const F MsF = (F)Ms;
        F z = 0, sM = 0, sH = 0, sMM = 0, sHH = 0, zA = 0, z2 = 0, z4 = 0;
        F dM = (F)(2 * mfirst - a.n - Ms);
        // FP64 chain: p_m = p_(m-1) qin[m] exp(2 h/T), one multiply instead of an exponential,
        // while the previous weight is at least 2^-964 (~6e-291) and the factor below 2^964
        // (~1.6e290); else, and for FP32, the exponential. <= 64 steps of a few ulp each keep p
        // within ~1e-13. The guards compare high words on the integer pipe (positive doubles
        // order like their bit patterns).
        const F R = (kChain && !by_warp) ? ex<F>((F)2 * hT) : (F)0;
        F pprev = 0;
        for (int m = mfirst; m < a.n_m; m += mstep, dM += dstep) {
            if (is_neg_inf(Lr[m])) { pprev = 0; continue; }
            F p;
            if constexpr (kChain) {
                const F f = by_warp ? (F)0 : qin[m] * R;
                p = (!by_warp && __double2hiint(pprev) >= 0x03b00000 && __double2hiint(f) < 0x7c300000)
                        ? pprev * f
                        : ex<F>(fmaF(hT, dM, Lr[m] - Ls));
            } else {
                p = ex<F>((Lr[m] - Ls) + (Llo[m] - Lls) + fmaF(hT, dM, hTlo * dM));
            }
            pprev = p;
            const F dH = fmaF(-hF, dM, mu[m] - mus);
            const F pM = p * dM, pH = p * dH;
            z += p;
            sM += pM;
            sH += pH;
            if (variances) {
                sMM += pM * dM;
                sHH += fmaF(p, var[m], pH * dH);
            }
            if (mag) {
                const F Mm = MsF + dM, M2 = Mm * Mm;
                zA += p * absF(Mm);
                z2 += p * M2;
                z4 += p * M2 * M2;
            }
        }
        if (by_warp) {
            F v[8] = {z, sM, sH, sMM, sHH, zA, z2, z4};
            warp_sum8(v);
            if (lane != 0) continue;
            z = v[0]; sM = v[1]; sH = v[2]; sMM = v[3]; sHH = v[4]; zA = v[5]; z2 = v[6]; z4 = v[7];
        }
        const F iz = (F)1 / z;
        const F dm = sM * iz, dh = sH * iz;
        const size_t o = (size_t)it * a.nh + ih;
        if (a.logZ) a.logZ[o] = L[ms] + hTd * (double)Ms + (double)lg<F>(z);
        if (a.E) a.E[o] = (double)(fmaF(-hF, MsF, mus) + dh);
        if (a.M) a.M[o] = (double)(MsF + dm);
        if (a.C) a.C[o] = (double)(fmaF(sHH, iz, -dh * dh) * invT2);
        if (a.chi) a.chi[o] = (double)(fmaF(sMM, iz, -dm * dm) * invT);
        if (mag) {
            const F m2 = z2 * iz, m4 = z4 * iz;
            if (a.absM) a.absM[o] = (double)(zA * iz);
            if (a.M2) a.M2[o] = (double)m2;
            if (a.M4) a.M4[o] = (double)m4;
            if (a.binder) a.binder[o] = m2 > (F)0 ? (double)((F)1 - m4 / ((F)3 * m2 * m2)) : 0.0;
        }
    }
}

// Fields all zero: the sum over M of Eq. (2) is the same at every temperature, so it is taken once
// per energy. The CTA first forms, for every energy bin e, G0(e) = sum_M g(e, M) and the lowest
// occupied bin, and the mean, variance, <|M|>, <M^2> and <M^4> of M within that bin, from exact integer sums (a
// flip-symmetric row has a mean of exactly zero). One warp per temperature then weighs
// the bins by w_e = G0(e) exp(-(E_e - E_0)/T), E_0 the lowest occupied energy (so w_e <= G0(e)
// and sum w <= 2^64): ln Z = -E_0/T + ln sum w, <H> = <E>,
// C = Var(E)/T^2 (two passes), <M> = sum w mu_e / sum w, chi = sum w (var_e + (mu_e - <M>)^2) /
// (T sum w), and the magnetisation moments from the bins' moments. Everything in double; one
// exponential per (temperature, energy) instead of one per (temperature, energy, M).
constexpr int kH0MaxE = 1024;            // energy bins whose moments fit the CTA's shared memory
constexpr int kH0Warps = 8;              // at most this many temperatures per CTA

// 128-bit integers to double (two roundings: within 2 ulp)
__device__ __forceinline__ double u128_to_double(unsigned __int128 x) {
    return (double)(uint64_t)(x >> 64) * 18446744073709551616.0 + (double)(uint64_t)x;
}
__device__ __forceinline__ double i128_to_double(__int128 x) {
    return x < 0 ? -u128_to_double((unsigned __int128)(-x)) : u128_to_double((unsigned __int128)x);
}

__global__ void __launch_bounds__(32 * kH0Warps) thermo_h0_kernel(const __grid_constant__ ThermoParams P) {
    const ThermoArgs& a = P.a;
    const double* Tv = a.T ? a.T : P.grid;
    extern __shared__ __align__(16) unsigned char sm[];
    double* G0v = reinterpret_cast<double*>(sm);      // configurations at energy e (as double)
    double* mu = G0v + a.n_e;
    double* vr = mu + a.n_e;
    double* ab = vr + a.n_e;
    double* q2 = ab + a.n_e;
    double* q4 = q2 + a.n_e;
    const int N = a.n, n_m = a.n_m;
    __shared__ int s_egs;                              // lowest energy bin with a configuration
    if (threadIdx.x == 0) s_egs = INT_MAX;
    __syncthreads();
    for (int e = threadIdx.x; e < a.n_e; e += blockDim.x) {
        // exact integer moments of the row (128-bit: c < 2^63, |M|^4 <= 2^24, at most 65 columns),
        // on the integer pipe; the variance about the integer Mp nearest the mean, also exact
        const int64_t* row = a.g + (size_t)e * n_m;
        unsigned __int128 G0 = 0, SA = 0, S2 = 0, S4 = 0;
        __int128 S1 = 0;
        for (int m = 0; m < n_m; ++m) {
            const uint64_t c = (uint64_t)row[m];
            if (!c) continue;
            const int M = 2 * m - N;
            const uint64_t aM = (uint64_t)(M < 0 ? -M : M), M2 = aM * aM;
            G0 += c;
            SA += (unsigned __int128)c * aM;
            S2 += (unsigned __int128)c * M2;
            S4 += (unsigned __int128)c * (M2 * M2);
            S1 += M < 0 ? -(__int128)((unsigned __int128)c * aM) : (__int128)((unsigned __int128)c * aM);
        }
        if (G0 == 0) {
            G0v[e] = 0;
            mu[e] = vr[e] = ab[e] = q2[e] = q4[e] = 0;
            continue;
        }
        atomicMin(&s_egs, e);
        const double G0d = u128_to_double(G0), inv = 1.0 / G0d, mean = i128_to_double(S1) * inv;
        const int64_t Mp = llrint(mean);
        const __int128 Q = (__int128)S2 - 2 * (__int128)Mp * S1 + (__int128)(Mp * Mp) * (__int128)G0;   // sum c (M - Mp)^2
        const double dm = mean - (double)Mp;                                                            // |dm| <= 1/2
        G0v[e] = G0d;
        mu[e] = mean;
        vr[e] = fmax(0.0, i128_to_double(Q) * inv - dm * dm);
        ab[e] = u128_to_double(SA) * inv;
        q2[e] = u128_to_double(S2) * inv;
        q4[e] = u128_to_double(S4) * inv;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    constexpr int kCache = 8;                          // weights kept in registers for the second pass
    const int egs = s_egs;
    for (int it = blockIdx.x * nw + warp; it < a.nT; it += gridDim.x * nw) {
        // weights relative to the lowest occupied energy E0: w(E) = g0(E) exp(-(E - E0)/T), at
        // most 1 per configuration, so Z exp(E0/T) = sum w <= 2^64 and ln Z = -E0/T + ln sum w
        const double invT = 1.0 / Tv[it];
        const double xmax = -(double)(a.e_min + 2 * egs) * invT;
        auto weight = [&](int e) { return G0v[e] == 0.0 ? 0.0 : G0v[e] * exp(-2.0 * (double)(e - egs) * invT); };
        double wc[kCache];
        double z = 0, sE = 0, sM = 0;
#pragma unroll
        for (int j = 0; j < kCache; ++j) {
            const int e = lane + 32 * j;
            wc[j] = e < a.n_e ? weight(e) : 0.0;
            if (e < a.n_e) {
                z += wc[j];
                sE += wc[j] * (double)(a.e_min + 2 * e);
                sM += wc[j] * mu[e];
            }
        }
        for (int e = lane + 32 * kCache; e < a.n_e; e += 32) {
            const double w = weight(e);
            z += w;
            sE += w * (double)(a.e_min + 2 * e);
            sM += w * mu[e];
        }
        z = warp_sum(z);
        sE = warp_sum(sE);
        sM = warp_sum(sM);
        const double iz = 1.0 / z, mE = sE * iz, mM = sM * iz;
        double vE = 0, vM = 0, sa = 0, s2 = 0, s4 = 0;
        auto add = [&](int e, double w) {
            const double dE = (double)(a.e_min + 2 * e) - mE, dM = mu[e] - mM;
            vE += w * dE * dE;
            vM += w * (vr[e] + dM * dM);
            sa += w * ab[e];
            s2 += w * q2[e];
            s4 += w * q4[e];
        };
#pragma unroll
        for (int j = 0; j < kCache; ++j)
            if (lane + 32 * j < a.n_e) add(lane + 32 * j, wc[j]);
        for (int e = lane + 32 * kCache; e < a.n_e; e += 32) add(e, weight(e));
        vE = warp_sum(vE);
        vM = warp_sum(vM);
        sa = warp_sum(sa);
        s2 = warp_sum(s2);
        s4 = warp_sum(s4);
        if (lane == 0)
            for (int ih = 0; ih < a.nh; ++ih) {         // every field of the grid is zero
                const size_t o = (size_t)it * a.nh + ih;
                if (a.logZ) a.logZ[o] = xmax + log(z);
                if (a.E) a.E[o] = mE;
                if (a.M) a.M[o] = mM;
                if (a.C) a.C[o] = vE * iz * invT * invT;
                if (a.chi) a.chi[o] = vM * iz * invT;
                const double m2 = s2 * iz, m4 = s4 * iz;
                if (a.absM) a.absM[o] = sa * iz;
                if (a.M2) a.M2[o] = m2;
                if (a.M4) a.M4[o] = m4;
                if (a.binder) a.binder[o] = m2 > 0 ? 1.0 - m4 / (3.0 * m2 * m2) : 0.0;
            }
    }
}

// The graph's energy sublattice in public bins: reachable energies E = e_lo + G k (k < n_e_c) sit
// at bins (E + S) / 2 = e0 + (G / 2) k.
void set_energy_sublattice(ThermoArgs& a, const isg_graph& g) {
    a.e0 = (int)((g.e_lo + g.S) / 2);
    a.eg = (int)(g.G / 2);
    a.n_on = (int)g.n_e_c;
}

// Enqueue the thermodynamics kernels; all pointers on the device. lng: n_e * n_m doubles, lngf:
// 2 * n_e * n_m floats of scratch. P.a.cluster is set here. h_zero: every field of the grid is 0
// (the per-energy path, which needs neither scratch array).
void launch_thermo(ThermoParams& P, double* lng, float* lngf, int precision, cudaStream_t s, bool h_zero) {
    ThermoArgs& a = P.a;
    if (h_zero && a.n_e <= kH0MaxE) {
        // every field zero: the per-energy path (thermo_h0_kernel), in double whatever the precision
        // few temperatures: fewer warps a CTA, so the per-temperature chains of double operations
        // spread over more SMs (each CTA forms the energies' moments on the integer pipe)
        a.cluster = 1;
        const int warps = std::max(1, std::min(kH0Warps, a.nT / device_info().sms));
        const int ctas = (a.nT + warps - 1) / warps;
        thermo_h0_kernel<<<ctas, 32 * warps, 6 * sizeof(double) * (size_t)a.n_e, s>>>(P);
        ISG_CUDA(cudaGetLastError());
        return;
    }
    const int nbins = a.n_e * a.n_m;
    float* lnglo = lngf + nbins;
    // 128 threads: one warp per SM sub-partition, so the FP64 logarithms of a small table spread
    // over as many FP64 units as there are warps
    log_counts_kernel<<<std::min(2048, (nbins + 127) / 128), 128, 0, s>>>(a.g, nbins, lng, lngf, lnglo);
    ISG_CUDA(cudaGetLastError());
    // Few temperatures (fewer than half the SMs): a cluster of up to 8 CTAs per temperature
    // shares stage 1's columns, one warp per column in each CTA. Fewer than the SMs: one CTA per
    // temperature, one warp per column. Otherwise 256 threads per CTA, several CTAs per SM.
    const int sms = device_info().sms;
    int csz = 1;
    if (2 * a.nT <= sms) csz = std::max(1, std::min(std::min(8, sms / a.nT), (a.n_m + 3) / 4));
    a.cluster = csz;
    const int cols = (a.n_m + csz - 1) / csz;
    const int threads = a.nT < sms ? 32 * std::min(32, std::max(8, cols)) : 256;
    const size_t smem = (size_t)a.n_m * (8 + 6 * (precision == ISG_FP64 ? sizeof(double) : sizeof(float)) + 4 + 4);
    auto launch = [&](auto kernel) {
        if (csz == 1) {
            kernel<<<a.nT, threads, smem, s>>>(P, lng, lngf, lnglo);
            return;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(a.nT * csz));
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)csz;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        ISG_CUDA(cudaLaunchKernelEx(&cfg, kernel, (const ThermoParams)P, (const double*)lng, (const float*)lngf,
                                    (const float*)lnglo));
    };
    if (precision == ISG_FP64) launch(thermo_kernel<double>);
    else launch(thermo_kernel<float>);
    ISG_CUDA(cudaGetLastError());
}

}  // namespace isg

using namespace isg;

extern "C" isg_status isg_specific_heat_peak(const int64_t* g, int32_t g_on_device, const isg_graph* graph, double h,
                                             double T_lo, double T_hi, int32_t precision, void* stream,
                                             double* T_peak, double* C_peak) {
    return guarded([&] {
        NvtxRange nvtx("isg_specific_heat_peak");
        if (!g || !graph || !T_peak) fail(ISG_ERR_INVALID, "NULL argument");
        if (!(T_lo > 0) || !(T_hi > T_lo) || !std::isfinite(T_hi) || !std::isfinite(h))
            fail(ISG_ERR_INVALID, "need 0 < T_lo < T_hi, finite, and a finite field");
        if (precision != ISG_FP64 && precision != ISG_FP32) fail(ISG_ERR_INVALID, "precision must be ISG_FP64 or ISG_FP32");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int n_m = graph->n + 1, n_e = (int)(graph->S + 1);
        const size_t gbytes = sizeof(int64_t) * (size_t)n_e * n_m;
        constexpr int kGrid = 257;                   // odd: the bracket keeps a centre point
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) & ~(size_t)255; return o; };
        const size_t o_lng = take(sizeof(double) * (size_t)n_e * n_m);
        const size_t o_lngf = take(2 * sizeof(float) * (size_t)n_e * n_m);
        const size_t o_g = g_on_device ? 0 : take(gbytes);
        const size_t o_C = take(sizeof(double) * kGrid);
        char* scratch = static_cast<char*>(scratch_alloc(off, s));
        struct Free {
            char* p; cudaStream_t s;
            ~Free() { if (p) cudaFreeAsync(p, s); }
        } guard{scratch, s};
        std::unique_ptr<ThermoParams> P(new ThermoParams());
        ThermoArgs& a = P->a;
        a.n = graph->n; a.n_e = n_e; a.n_m = n_m; a.nT = kGrid; a.nh = 1; a.e_min = -graph->S;
        set_energy_sublattice(a, *graph);
        a.T = nullptr;
        a.h = nullptr;
        if (g_on_device) a.g = g;
        else {
            ISG_CUDA(cudaMemcpyAsync(scratch + o_g, g, gbytes, cudaMemcpyHostToDevice, s));
            a.g = reinterpret_cast<int64_t*>(scratch + o_g);
        }
        a.C = reinterpret_cast<double*>(scratch + o_C);
        std::vector<double> C(kGrid);
        double lo = T_lo, hi = T_hi, best_T = T_lo, best_C = -1;
        // a uniform grid over the bracket, then the bracket shrinks to the two neighbours of the
        // best grid point, until it is narrower than 1e-12 of the temperature
        for (int round = 0; round < 12; ++round) {
            for (int k = 0; k < kGrid; ++k) P->grid[k] = lo + (hi - lo) * k / (kGrid - 1);
            P->grid[kGrid] = h;
            launch_thermo(*P, reinterpret_cast<double*>(scratch + o_lng), reinterpret_cast<float*>(scratch + o_lngf),
                          precision, s, h == 0.0);
            ISG_CUDA(cudaMemcpyAsync(C.data(), a.C, sizeof(double) * kGrid, cudaMemcpyDeviceToHost, s));
            ISG_CUDA(cudaStreamSynchronize(s));
            int kb = 0;
            for (int k = 1; k < kGrid; ++k) if (C[k] > C[kb]) kb = k;
            best_T = P->grid[kb];
            best_C = C[kb];
            const double step = (hi - lo) / (kGrid - 1);
            lo = std::max(T_lo, best_T - step);
            hi = std::min(T_hi, best_T + step);
            if (hi - lo < 1e-12 * best_T) break;
        }
        *T_peak = best_T;
        if (C_peak) *C_peak = best_C;
    });
}

// One evaluation of the grid T x h: validation, scratch, the kernels and the copies back. outs
// holds logZ, E, M, C, chi, absM, M2, M4, binder (any may be NULL).
static void thermo_grid(const int64_t* g, int32_t g_on_device, const isg_graph* graph, int32_t nT, const double* T,
                        int32_t nh, const double* h, int32_t precision, void* stream, int32_t out_on_device,
                        double* const outs_host[kThermoOuts]) {
    if (!g || !graph || !T || !h) fail(ISG_ERR_INVALID, "NULL argument");
    if (nT < 1 || nh < 1) fail(ISG_ERR_INVALID, "nT and nh must be >= 1");
    if (precision != ISG_FP64 && precision != ISG_FP32) fail(ISG_ERR_INVALID, "precision must be ISG_FP64 or ISG_FP32");
    for (int i = 0; i < nT; ++i)
        if (!(T[i] > 0) || !std::isfinite(T[i])) fail(ISG_ERR_INVALID, "temperatures must be finite and > 0");
    for (int i = 0; i < nh; ++i)
        if (!std::isfinite(h[i])) fail(ISG_ERR_INVALID, "fields must be finite");
    if (graph->S > (1 << 24)) fail(ISG_ERR_TOO_LARGE, "energy range too large for the thermodynamics kernels");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n_m = graph->n + 1, n_e = (int)(graph->S + 1);
    const size_t gbytes = sizeof(int64_t) * (size_t)n_e * n_m;
    const size_t pts = (size_t)nT * nh;
    int n_out = 0;
    for (int k = 0; k < kThermoOuts; ++k) n_out += outs_host[k] != nullptr;
    // scratch: [lng][lngf, lnglo][T][h][g copy if host][requested outputs if host]
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) & ~(size_t)255; return o; };
    const size_t o_lng = take(sizeof(double) * (size_t)n_e * n_m);
    const size_t o_lngf = take(2 * sizeof(float) * (size_t)n_e * n_m);
    const bool inline_grid = nT + nh <= kInlineGrid;
    const size_t o_T = inline_grid ? 0 : take(sizeof(double) * nT), o_h = inline_grid ? 0 : take(sizeof(double) * nh);
    const size_t o_g = g_on_device ? 0 : take(gbytes);
    const size_t o_out = out_on_device ? 0 : take(n_out * sizeof(double) * pts);
    char* scratch = static_cast<char*>(scratch_alloc(off, s));
    struct Free {
        char* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } guard{scratch, s};
    std::unique_ptr<ThermoParams> P(new ThermoParams());
    ThermoArgs& a = P->a;
    a.n = graph->n; a.n_e = n_e; a.n_m = n_m; a.nT = nT; a.nh = nh; a.e_min = -graph->S;
    set_energy_sublattice(a, *graph);
    if (inline_grid) {
        std::memcpy(P->grid, T, sizeof(double) * nT);
        std::memcpy(P->grid + nT, h, sizeof(double) * nh);
        a.T = nullptr;
        a.h = nullptr;
    } else {
        a.T = reinterpret_cast<double*>(scratch + o_T);
        a.h = reinterpret_cast<double*>(scratch + o_h);
        ISG_CUDA(cudaMemcpyAsync(scratch + o_T, T, sizeof(double) * nT, cudaMemcpyHostToDevice, s));
        ISG_CUDA(cudaMemcpyAsync(scratch + o_h, h, sizeof(double) * nh, cudaMemcpyHostToDevice, s));
    }
    // host buffers go through one pinned stage: [g][requested outputs]
    std::unique_ptr<PinnedStage> stage;
    if (!g_on_device || !out_on_device)
        stage.reset(new PinnedStage((g_on_device ? 0 : gbytes) + (out_on_device ? 0 : n_out * sizeof(double) * pts), s));
    if (g_on_device) a.g = g;
    else {
        std::memcpy(stage->data(), g, gbytes);
        ISG_CUDA(cudaMemcpyAsync(scratch + o_g, stage->data(), gbytes, cudaMemcpyHostToDevice, s));
        a.g = reinterpret_cast<int64_t*>(scratch + o_g);
    }
    double* outs_dev[kThermoOuts];
    for (int k = 0, j = 0; k < kThermoOuts; ++k)
        outs_dev[k] = !outs_host[k] ? nullptr
                      : out_on_device ? outs_host[k]
                                      : reinterpret_cast<double*>(scratch + o_out) + (j++) * pts;
    a.logZ = outs_dev[0]; a.E = outs_dev[1]; a.M = outs_dev[2]; a.C = outs_dev[3]; a.chi = outs_dev[4];
    a.absM = outs_dev[5]; a.M2 = outs_dev[6]; a.M4 = outs_dev[7]; a.binder = outs_dev[8];
    bool h_zero = true;
    for (int k = 0; k < nh; ++k) h_zero = h_zero && h[k] == 0.0;
    launch_thermo(*P, reinterpret_cast<double*>(scratch + o_lng), reinterpret_cast<float*>(scratch + o_lngf), precision, s,
                  h_zero);
    if (!out_on_device) {
        // the requested outputs lie side by side in the scratch: one copy into the stage
        char* out_host = stage->data() + (g_on_device ? 0 : gbytes);
        ISG_CUDA(cudaMemcpyAsync(out_host, scratch + o_out, n_out * sizeof(double) * pts, cudaMemcpyDeviceToHost, s));
        ISG_CUDA(cudaStreamSynchronize(s));
        stage->synced();
        for (int k = 0, j = 0; k < kThermoOuts; ++k)
            if (outs_host[k]) std::memcpy(outs_host[k], out_host + (j++) * sizeof(double) * pts, sizeof(double) * pts);
    } else if (!g_on_device) {
        ISG_CUDA(cudaStreamSynchronize(s));
        stage->synced();
    }
}

extern "C" isg_status isg_thermo(const int64_t* g, int32_t g_on_device, const isg_graph* graph, int32_t nT,
                                 const double* T, int32_t nh, const double* h, int32_t precision, void* stream,
                                 int32_t out_on_device, double* logZ, double* E, double* M, double* C, double* chi) {
    return guarded([&] {
        NvtxRange nvtx("isg_thermo");
        double* const outs[kThermoOuts] = {logZ, E, M, C, chi, nullptr, nullptr, nullptr, nullptr};
        thermo_grid(g, g_on_device, graph, nT, T, nh, h, precision, stream, out_on_device, outs);
    });
}

extern "C" isg_status isg_magnetisation(const int64_t* g, int32_t g_on_device, const isg_graph* graph, int32_t nT,
                                        const double* T, int32_t nh, const double* h, int32_t precision,
                                        void* stream, int32_t out_on_device, double* abs_M, double* M2, double* M4,
                                        double* binder) {
    return guarded([&] {
        NvtxRange nvtx("isg_magnetisation");
        double* const outs[kThermoOuts] = {nullptr, nullptr, nullptr, nullptr, nullptr, abs_M, M2, M4, binder};
        thermo_grid(g, g_on_device, graph, nT, T, nh, h, precision, stream, out_on_device, outs);
    });
}
