// Velocity sets, link-mask layout and population storage of the sm_103a lattice Boltzmann
// kernels (Tsompanas et al., arXiv 1802.07525, Sec. 3.1).
//
// D2Q9 follows Eqs. 1-3 and the weights of Eqs. 6-8; the order of c5..c8 is the one fixed by the
// bounce-back pairs of Eq. 11 (5<->7, 2<->4, 6<->8).  D3Q19 (3-D flow) has the rest velocity, six
// faces and twelve edges with opposites adjacent; D2Q5 / D3Q7 carry the substrate (Eq. 12) with
// the linear equilibrium, and, as the text after Eq. 12 has it, D2Q9 with the equilibrium of
// Eq. 5 (C in place of rho) is the paper-literal alternative in 2-D.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace mfc {

enum : int { BC_WALL = 0, BC_PERIODIC = 1, BC_INOUT = 2 };
enum : uint8_t { CLS_FLOW = 1, CLS_ADE = 2, CLS_SINK = 4 };

// ---- velocity sets ---------------------------------------------------------------------------

template <int DIM> struct FlowSet;
// Transport velocity set: AQ = 5 (D2Q5) or 9 (D2Q9, quadratic equilibrium) in 2-D, 7 in 3-D.
template <int DIM> __host__ __device__ constexpr int default_aq() { return DIM == 2 ? 5 : 7; }
template <int DIM, int AQ = default_aq<DIM>()> struct AdeSet;

template <> struct FlowSet<2> {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        constexpr int t[9][3] = {{0, 0, 0}, {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
                                 {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
        return t[i][a];
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[i];
    }
    __host__ __device__ static constexpr float w(int i)
    {
        return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
    }
    __host__ __device__ static constexpr double wd(int i)
    {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <> struct FlowSet<3> {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return t[i][a];
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
    __host__ __device__ static constexpr float w(int i)
    {
        return i == 0 ? 1.0f / 3.0f : (i < 7 ? 1.0f / 18.0f : 1.0f / 36.0f);
    }
    __host__ __device__ static constexpr double wd(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

template <> struct AdeSet<2, 5> {
    static constexpr int Q = 5;
    static constexpr bool quadratic = false;  // G_i^eq = w_i C (1 + c_i.u / cs^2)
    static constexpr float inv_cs2 = 3.0f;  // D = (tau_c - 1/2) / 3
    __host__ __device__ static constexpr int c(int i, int a) { return FlowSet<2>::c(i, a); }
    __host__ __device__ static constexpr int opp(int i) { return FlowSet<2>::opp(i); }
    __host__ __device__ static constexpr float w(int i) { return i == 0 ? 1.0f / 3.0f : 1.0f / 6.0f; }
    __host__ __device__ static constexpr double wd(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
};

template <> struct AdeSet<3, 7> {
    static constexpr int Q = 7;
    static constexpr bool quadratic = false;
    static constexpr float inv_cs2 = 4.0f;  // D = (tau_c - 1/2) / 4
    __host__ __device__ static constexpr int c(int i, int a) { return FlowSet<3>::c(i, a); }
    __host__ __device__ static constexpr int opp(int i) { return FlowSet<3>::opp(i); }
    __host__ __device__ static constexpr float w(int i) { return i == 0 ? 1.0f / 4.0f : 1.0f / 8.0f; }
    __host__ __device__ static constexpr double wd(int i) { return i == 0 ? 1.0 / 4.0 : 1.0 / 8.0; }
};

// D2Q9 transport with the flow equilibrium of Eq. 5 (C in place of rho):
// G_i^eq = w_i C (1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u); D = (tau_c - 1/2) / 3.
template <> struct AdeSet<2, 9> {
    static constexpr int Q = 9;
    static constexpr bool quadratic = true;
    static constexpr float inv_cs2 = 3.0f;
    __host__ __device__ static constexpr int c(int i, int a) { return FlowSet<2>::c(i, a); }
    __host__ __device__ static constexpr int opp(int i) { return FlowSet<2>::opp(i); }
    __host__ __device__ static constexpr float w(int i) { return FlowSet<2>::w(i); }
    __host__ __device__ static constexpr double wd(int i) { return FlowSet<2>::wd(i); }
};

// Weight w_i of a velocity set in the arithmetic type R: the FP32 constants in FP32 arithmetic,
// the rationals rounded once to double in FP64 arithmetic.
template <typename SET, typename R> __host__ __device__ constexpr R weight(int i)
{
    return std::is_same<R, double>::value ? (R)SET::wd(i) : (R)SET::w(i);
}

// ---- link masks ------------------------------------------------------------------------------
// One word per node.  Bit 0: the node is blocked for the flow.  Bit i (1..Qf-1): the flow
// population arriving along c_i bounces back (its source is a wall or a blocked node).
// Bit Qf: blocked for transport.  Bit Qf+i (1..Qa-1): the transport population along c_i
// bounces back.  Bit Qf+Qa: consumption node.  16-bit words when they fit (D2Q9 + D2Q5), else 32.
template <int DIM, int AQ = default_aq<DIM>()> struct Links {
    static constexpr int QF = FlowSet<DIM>::Q;
    static constexpr int QA = AdeSet<DIM, AQ>::Q;
    static constexpr int FLOW_SELF = 0;
    static constexpr int ADE_SELF = QF;
    static constexpr int SINK = QF + QA;
    using T = typename std::conditional<(QF + QA < 16), uint16_t, uint32_t>::type;
};

// ---- storage ---------------------------------------------------------------------------------
// Populations are stored as deviations from the rest state in FP32 or FP16 with FP32
// arithmetic, or in FP64 with FP64 arithmetic (the double-precision instantiation of the same
// kernels, for parity with the FP64 reference at rounding level).  Arith<ST>::T is the type of
// the arithmetic, of the fields (rho - 1, u, C - c_ref) and of the per-node check-step terms.
template <typename ST> struct Arith {
    using T = float;
};
template <> struct Arith<double> {
    using T = double;
};
__device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st(double *p, double v) { *p = v; }
// The value a store of v keeps (identity in FP32 and FP64, rounded to FP16 in FP16 storage).
__device__ __forceinline__ float kept(const float *, float v) { return v; }
__device__ __forceinline__ float kept(const __half *, float v) { return __half2float(__float2half_rn(v)); }
__device__ __forceinline__ double kept(const double *, double v) { return v; }
// 1 / x: the fast FP32 reciprocal-division (at most 2 ulp) in FP32, IEEE division in FP64.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Sums produced by a residual-check step (one double each, per block then per lattice).
enum : int {
    SUM_DU2 = 0,    // sum |u^n - u^(n-1)|^2 over flow-open nodes
    SUM_U2 = 1,     // sum |u^n|^2
    SUM_MASS = 2,   // sum rho
    SUM_DC2 = 3,    // sum (C^n - C^(n-1))^2 over transport-open nodes
    SUM_C2 = 4,     // sum C^2
    SUM_C = 5,      // sum C
    SUM_CURRENT = 6,// sum over consumption nodes of the consumption (k C, or k C K_s / (K_s + C))
    SUM_BAD = 7,    // count of non-finite values
    SUM_FAST = 8,   // count of flow-open nodes outside the scheme's range: |u|^2 >= cs^2 = 1/3
                    // (the flow at or above the lattice sound speed) or rho <= 0
    NSUM = 9
};

// Per-lattice results written by the finalize kernel: the sums, then the two residuals.
enum : int { RES_FLOW = NSUM, RES_ADE = NSUM + 1, NRESULT = NSUM + 2 };

}  // namespace mfc
