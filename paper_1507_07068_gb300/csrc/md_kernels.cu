// md_kernels.cu -- the sm_103a kernels of libmd and their launchers.
//
// Per time step (Fig. 5 / Table 1 of Pal et al., arXiv:1507.07068):
//   k_decide    Task 1 decision (Sec. 2.6 skin/2 rule on max_i |x_i - x_build,i|, reduced by
//               the drift that made the positions) -> device flag + graph conditional; Task 2
//               (the indenter moves by v dt); advances the position-buffer counter
//   [rebuild]   Task 1 rebuild: k_bin (wrap, FP64 cell keys, histogram), scan, k_scatter,
//               k_cellsort (ascending caller id within a cell), k_gather/k_copyback
//               (permute every per-atom array), k_nbr (full Cr-Cr Verlet list), k_nbrc /
//               k_nbrc_near (Cr-C list through the indenter's own cell grid), k_build_done
//   k_verlet1   Task 3 (half kick + drift, Eqs. A11-A12, the FP32 cell-relative positions,
//               the displacement tests) into the other position buffer: every step in FP64;
//               in mixed precision only after a list build (the force epilogue drifts)
//   k_density   Task 4a: rho_i, P_i (Eq. A2) -> F'(rho_i), M'(P_i), F(rho_i), M(P_i) (Eq. A3);
//               rebuilds the inner list (Sec. 2.6) when its own displacement test asks
//   k_morse_mixed  Task 4c for the atoms under the indenter (one warp per atom)
//   k_force     Task 4b,c + 5: Eq. (1) with the M term (A6-A8, A10), Morse (A5, A9),
//               indenter load; epilogue: closing half kick (Task 5) and, in mixed
//               precision, the next step's Task 3
//   k_reduce    per-replica FP64 sums of the CTA partials in a fixed order (once per call)
// Outside the step: k_state_prep / k_state_scan / k_state_need (md_set_state),
// k_drift_prep (the drift made by a force evaluation outside a step), k_virial_* (per-atom
// virial), the allocation-free small-system kernels (md_forces_small).
// Every per-atom kernel writes only its own atom (full neighbour list: no atomics in
// the force path); energy and load sums are warp-shuffle -> CTA partial -> fixed-order
// final pass, so results do not depend on scheduling.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "md_internal.h"

#define MD_UNROLL 4   // neighbour entries per lane whose loads are issued together
#define MD_SORT_MAX 2048     // largest cell k_cellsort orders

// ============================================================================ host:
// potential forms used to fill the tables (FP64), restated from the Appendix.

namespace {

// Knot values are evaluated in extended precision and rounded once to FP64: the slope of
// a Hermite cubic carries knot-value rounding amplified by 1.5/h, so once-rounded knots
// keep the FP64 tables reproducible to the last bit.
struct HostPot {
    md_params p;
    long double f_rc = 0, df_rc = 0, m_rc = 0, dm_rc = 0;
    long double e[4];   // Eq. A4 about x = d: Phi = t^2 (e0 + e1 t + e2 t^2 + e3 t^3), t = r/r_e - d

    long double f_raw(long double r) const { return (long double)p.f_e * powl((long double)p.r_e / r, (long double)p.beta); }
    long double df_raw(long double r) const { return -(long double)p.beta * f_raw(r) / r; }
    void morse_raw(long double y, long double &v, long double &dv) const {
        long double E = expl(-0.5L * (long double)p.alpha_x * (y / (long double)p.y_eq - 1.0L));
        v = (long double)p.D_o * E * (E - 2.0L);
        dv = -(long double)p.D_o * (long double)p.alpha_x / (long double)p.y_eq * E * (E - 1.0L);
    }
    void f(long double r, long double &v, long double &dv) const {   // r < rc branch
        v = f_raw(r) - f_rc - (r - (long double)p.rc) * df_rc;
        dv = df_raw(r) - df_rc;
    }
    void phi(long double r, long double &v, long double &dv) const {
        long double t = r / (long double)p.r_e - (long double)p.d;
        if (t > 0.0L) { v = dv = 0.0L; return; }
        v = t * t * (e[0] + t * (e[1] + t * (e[2] + t * e[3])));
        dv = t * (2.0L * e[0] + t * (3.0L * e[1] + t * (4.0L * e[2] + t * 5.0L * e[3]))) / (long double)p.r_e;
    }
    void morse(long double y, long double &v, long double &dv) const {
        morse_raw(y, v, dv);
        v -= m_rc + (y - (long double)p.rc_morse) * dm_rc;
        dv -= dm_rc;
    }
};

// cubic on [0,1) from end values g0, g1 and end slopes (per unit t) m0, m1
void hermite_coeffs(double g0, double g1, double m0, double m1, Cf64 &c)
{
    c.x = g0;
    c.y = m0;
    c.z = 3.0 * (g1 - g0) - 2.0 * m0 - m1;
    c.w = 2.0 * (g0 - g1) + m0 + m1;
}

template <class Fn>
void fill_table(int n, double r0, double r1, Fn g, std::vector<Cf64> &out)
{
    out.resize(n);
    double h = (r1 - r0) / n;
    std::vector<double> v(n + 1), d(n + 1);
    for (int k = 0; k <= n; ++k) {
        double r = (k == n) ? r1 : r0 + k * h;   // host code is built without FMA contraction
        long double vl, dl;
        g((long double)r, vl, dl);
        v[k] = (double)vl;
        d[k] = (double)dl;
    }
    for (int k = 0; k < n; ++k) hermite_coeffs(v[k], v[k + 1], d[k] * h, d[k + 1] * h, out[k]);
}

}  // namespace

// The analytic forms of md_params in FP64 (Eqs. A2-A5, shifted-force constants, Eq. A4 in
// its Taylor form about the double root): the fields that md_build_pot and md_pot_forms share.
static void fill_forms(const md_params *p, PotDev *P, HostPot &H)
{
    H.p = *p;
    // Taylor coefficients of the cubic of Eq. A4 about x = d
    const long double a0 = p->a[0], a1 = p->a[1], a2 = p->a[2], a3 = p->a[3], d = p->d;
    H.e[0] = ((a3 * d + a2) * d + a1) * d + a0;
    H.e[1] = (3.0L * a3 * d + 2.0L * a2) * d + a1;
    H.e[2] = 3.0L * a3 * d + a2;
    H.e[3] = a3;
    if (p->shifted) {
        H.f_rc = H.f_raw(p->rc);
        H.df_rc = H.df_raw(p->rc);
        H.morse_raw(p->rc_morse, H.m_rc, H.dm_rc);
    }
    P->f_e = p->f_e; P->r_e = p->r_e; P->beta = p->beta;
    P->lf0 = log2(p->f_e) + p->beta * log2(p->r_e);
    P->F_o = p->F_o; P->n = p->n; P->rho_e = p->rho_e; P->alpha = p->alpha; P->P_e = p->P_e;
    for (int k = 0; k < 4; ++k) P->b[k] = (double)H.e[k];
    P->d = p->d;
    P->D_o = p->D_o; P->half_ax = 0.5 * p->alpha_x; P->inv_yeq = 1.0 / p->y_eq;
    P->rc = p->rc; P->rc_m = p->rc_morse; P->rc2 = p->rc * p->rc; P->rcm2 = p->rc_morse * p->rc_morse;
    P->f_rc = (double)H.f_rc; P->df_rc = (double)H.df_rc; P->m_rc = (double)H.m_rc; P->dm_rc = (double)H.dm_rc;
    P->shifted = p->shifted;
}

int md_build_pot(const md_params *p, PotDev *P, Cf64 **d_tabs64, float4 **d_tabs32, char *err, size_t errlen)
{
    memset(P, 0, sizeof(*P));
    if (!(p->r_e > 0 && p->f_e > 0 && p->rho_e > 0 && p->P_e > 0 && p->y_eq > 0 && p->rc > 0 &&
          p->rc_morse > 0 && p->r_min > 0 && p->r_min < p->rc && p->r_min < p->rc_morse && p->h > 0)) {
        snprintf(err, errlen, "md_params: r_e, f_e, rho_e, P_e, y_eq, rc, rc_morse, h must be > 0 and r_min < both cut-offs");
        return MD_ERR_ARG;
    }
    HostPot H;
    fill_forms(p, P, H);
    P->tabulated = p->tabulated;
    P->r_min = p->r_min;
    int nf = (int)ceil((p->rc - p->r_min) / p->h - 1e-9);
    int nm = (int)ceil((p->rc_morse - p->r_min) / p->h - 1e-9);
    if (nf < 1) nf = 1;
    if (nm < 1) nm = 1;
    if (nf > (1 << 24) || nm > (1 << 24)) { snprintf(err, errlen, "md_params: table spacing h too small"); return MD_ERR_ARG; }
    P->nf = nf; P->nm = nm;
    P->inv_hf = nf / (p->rc - p->r_min);
    P->inv_hm = nm / (p->rc_morse - p->r_min);
    *d_tabs64 = nullptr; *d_tabs32 = nullptr;
    std::vector<Cf64> tf, tp, tm;
    fill_table(nf, p->r_min, p->rc, [&](long double r, long double &v, long double &dv) { H.f(r, v, dv); }, tf);
    fill_table(nf, p->r_min, p->rc, [&](long double r, long double &v, long double &dv) { H.phi(r, v, dv); }, tp);
    fill_table(nm, p->r_min, p->rc_morse, [&](long double r, long double &v, long double &dv) { H.morse(r, v, dv); }, tm);
    size_t ntot = (size_t)4 * nf + nm;   // FP64: f, Phi, Morse (+ unused); FP32 adds f/Phi interleaved
    std::vector<Cf64> all;
    all.reserve(ntot);
    all.insert(all.end(), tf.begin(), tf.end());
    all.insert(all.end(), tp.begin(), tp.end());
    all.insert(all.end(), tm.begin(), tm.end());
    std::vector<float4> all32(ntot);
    for (size_t k = 0; k < (size_t)2 * nf + nm; ++k)
        all32[k] = make_float4((float)all[k].x, (float)all[k].y, (float)all[k].z, (float)all[k].w);
    for (int k = 0; k < nf; ++k) {
        all32[2 * nf + nm + 2 * k] = all32[k];
        all32[2 * nf + nm + 2 * k + 1] = all32[nf + k];
    }
    all.resize(ntot);
    if (cudaMalloc(d_tabs64, ntot * sizeof(Cf64)) != cudaSuccess ||
        cudaMalloc(d_tabs32, ntot * sizeof(float4)) != cudaSuccess) {
        snprintf(err, errlen, "cudaMalloc of potential tables failed");
        if (*d_tabs64) cudaFree(*d_tabs64);
        *d_tabs64 = nullptr;
        return MD_ERR_CUDA;
    }
    if (cudaMemcpy(*d_tabs64, all.data(), ntot * sizeof(Cf64), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(*d_tabs32, all32.data(), ntot * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess) {
        snprintf(err, errlen, "copy of potential tables failed");
        return MD_ERR_CUDA;
    }
    P->tf = *d_tabs64; P->tp = *d_tabs64 + nf; P->tm = *d_tabs64 + 2 * nf;
    P->tf32 = *d_tabs32; P->tp32 = *d_tabs32 + nf; P->tm32 = *d_tabs32 + 2 * nf;
    PotF32 &q = P->q;
    q.inv_hf = (float)P->inv_hf; q.rmin_s_f = (float)(P->r_min * P->inv_hf);
    q.inv_hm = (float)P->inv_hm; q.rmin_s_m = (float)(P->r_min * P->inv_hm);
    q.lf0 = (float)P->lf0; q.beta = (float)P->beta; q.f_rc = (float)P->f_rc; q.df_rc = (float)P->df_rc;
    q.rc = (float)P->rc; q.inv_re = (float)(1.0 / P->r_e); q.d = (float)P->d;
    {
        // Eq. A4 about t = tc: rs = r_e (d + tc) is the FP32 number nearest 0.95 r_e (between
        // BCC's first two neighbour shells for the forms here), so that r - rs is exact near
        // the first shells.  The cubics B(t) = sum e_k t^k (Phi = t^2 B) and
        // C(t) = sum (k + 2) e_k t^k / r_e (dPhi/dr = t C) are re-expanded in s = t - tc in
        // extended precision and rounded once.
        const float rs = (float)(0.95L * (long double)p->r_e);
        const long double re = p->r_e;
        const long double tc = (long double)rs / re - (long double)p->d;
        long double B[4], Cc[4];
        for (int k = 0; k < 4; ++k) { B[k] = H.e[k]; Cc[k] = (k + 2) * H.e[k] / re; }
        auto shift = [&](const long double (&c)[4], float (&o)[4]) {
            o[0] = (float)(((c[3] * tc + c[2]) * tc + c[1]) * tc + c[0]);
            o[1] = (float)((3.0L * c[3] * tc + 2.0L * c[2]) * tc + c[1]);
            o[2] = (float)(3.0L * c[3] * tc + c[2]);
            o[3] = (float)c[3];
        };
        float bb[4], cc[4];
        shift(B, bb);
        shift(Cc, cc);
        q.b0 = bb[0]; q.b1 = bb[1]; q.b2 = bb[2]; q.b3 = bb[3];
        q.c0 = cc[0]; q.c1 = cc[1]; q.c2 = cc[2]; q.c3 = cc[3];
        q.tc = (float)tc;
        q.rs = rs;
    }
    q.D_o = (float)P->D_o; q.half_ax = (float)P->half_ax; q.inv_yeq = (float)P->inv_yeq;
    q.m_rc = (float)P->m_rc; q.dm_rc = (float)P->dm_rc; q.rc_m = (float)P->rc_m;
    q.F_o = (float)P->F_o; q.n = (float)P->n; q.inv_rho_e = (float)(1.0 / P->rho_e); q.alpha = (float)P->alpha;
    q.inv_P_e = (float)(1.0 / P->P_e); q.rc2 = (float)P->rc2;
    q.tabulated = P->tabulated; q.nf = nf; q.nm = nm; q.tf = P->tf32; q.tp = P->tp32; q.tm = P->tm32;
    q.tfp = *d_tabs32 + 2 * nf + nm;
    const double half_beta = 0.5 * p->beta;
    q.ipow = (half_beta == floor(half_beta) && half_beta >= 1.0 && half_beta <= 8.0) ? (int)half_beta : 0;
    q.re2f = (float)(powl((long double)p->f_e, q.ipow > 0 ? 1.0L / q.ipow : 1.0L) * (long double)p->r_e * p->r_e);
    q.cf = (float)(H.f_rc - (long double)p->rc * H.df_rc);
    return MD_OK;
}

// ============================================================================ device helpers

namespace {

__device__ __forceinline__ int pack_cell(int c0, int c1, int c2)
{
    return c0 | (c1 << MD_CELL_BITS) | (c2 << (2 * MD_CELL_BITS));
}
__device__ __forceinline__ int cell_x(int p) { return p & ((1 << MD_CELL_BITS) - 1); }
__device__ __forceinline__ int cell_y(int p) { return (p >> MD_CELL_BITS) & ((1 << MD_CELL_BITS) - 1); }
__device__ __forceinline__ int cell_z(int p) { return (p >> (2 * MD_CELL_BITS)) & ((1 << MD_CELL_BITS) - 1); }

// a fixed-point length (units of qu = 2^-k A) in A, FP32: one rounding (the scaling is exact)
__device__ __forceinline__ float qf(int q, float qu) { return __int2float_rn(q) * qu; }

// ---- exact FP64 geometry of the list build and the skin test: every operation is a
// separately rounded IEEE operation (no FMA contraction), so cell keys and neighbour
// sets are reproducible on any IEEE machine from the same positions.
// floor(RN(d / w)) without the FP64 divide on the common path: q = d * (1/w) is within
// 3.4e-16 |q| of RN(d / w); when |q| < 1e6 and its fractional part is farther than 1e-9
// from an integer, both have the same floor.  Otherwise the divide decides.
__device__ __forceinline__ double floor_quot(double d, double w, double iw)
{
    const double q = __dmul_rn(d, iw);
    const double t = floor(q);
    const double f = __dsub_rn(q, t);
    if (fabs(q) < 1.0e6 && f > 1.0e-9 && f < 1.0 - 1.0e-9) return t;
    return floor(__ddiv_rn(d, w));
}
__device__ __forceinline__ double wrap_exact(double x, double lo, double L, double iL)
{
    const double m = floor_quot(__dsub_rn(x, lo), L, iL);
    return __dsub_rn(x, __dmul_rn(m, L));
}
__device__ __forceinline__ int cell_exact(double x, double lo, double w, double iw, int n)
{
    const double t = floor_quot(__dsub_rn(x, lo), w, iw);
    if (!(t >= 0.0)) return 0;
    if (t > (double)(n - 1)) return n - 1;
    return (int)t;
}
__device__ __forceinline__ double mi_exact(double d, int per, double L)
{
    if (per) {
        double half = 0.5 * L;
        if (d > half) d = __dsub_rn(d, L);
        else if (d < -half) d = __dadd_rn(d, L);
    }
    return d;
}
__device__ __forceinline__ double norm2_exact(double dx, double dy, double dz)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ---- potential, FP64
__device__ __forceinline__ void cubic64(const Cf64 *T, int n, double s, double inv_h, double &v, double &dv)
{
    double kf = fmin(fmax(floor(s), 0.0), (double)(n - 1));
    double t = s - kf;
    Cf64 c = T[(int)kf];
    v = fma(fma(fma(c.w, t, c.z), t, c.y), t, c.x);
    dv = fma(fma(3.0 * c.w, t, 2.0 * c.z), t, c.y) * inv_h;
}
__device__ __forceinline__ void f_64(const PotDev &P, double r, double &v, double &dv)
{
    if (P.tabulated) { cubic64(P.tf, P.nf, (r - P.r_min) * P.inv_hf, P.inv_hf, v, dv); return; }
    double fr = exp2(P.lf0 - P.beta * log2(r));
    v = fr - P.f_rc - (r - P.rc) * P.df_rc;
    dv = -P.beta * fr / r - P.df_rc;
}
__device__ __forceinline__ void phi_64(const PotDev &P, double r, double &v, double &dv)
{
    if (P.tabulated) { cubic64(P.tp, P.nf, (r - P.r_min) * P.inv_hf, P.inv_hf, v, dv); return; }
    double t = r / P.r_e - P.d;
    if (t > 0.0) { v = dv = 0.0; return; }
    v = t * t * fma(fma(fma(P.b[3], t, P.b[2]), t, P.b[1]), t, P.b[0]);
    dv = t * fma(fma(fma(5.0 * P.b[3], t, 4.0 * P.b[2]), t, 3.0 * P.b[1]), t, 2.0 * P.b[0]) / P.r_e;
}
__device__ __forceinline__ void morse_64(const PotDev &P, double y, double &v, double &dv)
{
    if (P.tabulated) { cubic64(P.tm, P.nm, (y - P.r_min) * P.inv_hm, P.inv_hm, v, dv); return; }
    double E = exp(-P.half_ax * (y * P.inv_yeq - 1.0));
    v = P.D_o * E * (E - 2.0) - P.m_rc - (y - P.rc_m) * P.dm_rc;
    dv = -2.0 * P.D_o * P.half_ax * P.inv_yeq * E * (E - 1.0) - P.dm_rc;
}
// Eq. A3: F and F' (F' = F_o n^2 s^n ln s / rho), M and M' (M' = (2 alpha/P_e) u (1-u^2) e^{-u^2})
__device__ __forceinline__ void embed_64(const PotDev &P, double rho, double &F, double &Fp)
{
    if (!(rho > 0.0)) { F = Fp = 0.0; return; }
    double L = log(rho / P.rho_e);
    double sn = exp(P.n * L);
    F = -P.F_o * (1.0 - P.n * L) * sn;
    Fp = P.F_o * P.n * P.n * sn * L / rho;
}
__device__ __forceinline__ void mterm_64(const PotDev &P, double Ps, double &M, double &Mp)
{
    if (!(Ps > 0.0)) { M = Mp = 0.0; return; }
    double u = Ps / P.P_e - 1.0;
    double e = exp(-u * u);
    M = P.alpha * u * u * e;
    Mp = 2.0 * P.alpha / P.P_e * u * (1.0 - u * u) * e;
}

// ---- potential, FP32 (mixed precision)
__device__ __forceinline__ void cubic32(const float4 *T, int n, float s, float inv_h, float &v, float &dv)
{
    float kf = fminf(fmaxf(floorf(s), 0.0f), (float)(n - 1));
    float t = s - kf;
    float4 c = __ldg(&T[(int)kf]);
    v = fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
    dv = fmaf(fmaf(3.0f * c.w, t, 2.0f * c.z), t, c.y) * inv_h;
}

struct Pot32 : PotF32 {   // the FP32 constants (filled on the host) with the FP32 forms
    __device__ __forceinline__ void morse(float y, float &v, float &dv) const
    {
        if (tabulated) { cubic32(tm, nm, fmaf(y, inv_hm, -rmin_s_m), inv_hm, v, dv); return; }
        float E = expf(-half_ax * fmaf(y, inv_yeq, -1.0f));
        v = D_o * E * (E - 2.0f) - m_rc - (y - rc_m) * dm_rc;
        dv = -2.0f * D_o * half_ax * inv_yeq * E * (E - 1.0f) - dm_rc;
    }
    __device__ __forceinline__ void embed(float rho, float &F, float &Fp) const
    {
        if (!(rho > 0.0f)) { F = Fp = 0.0f; return; }
        float L = logf(rho * inv_rho_e);
        float sn = expf(n * L);
        F = -F_o * (1.0f - n * L) * sn;
        Fp = F_o * n * n * sn * L / rho;
    }
    __device__ __forceinline__ void mterm(float Ps, float &M, float &Mp) const
    {
        if (!(Ps > 0.0f)) { M = Mp = 0.0f; return; }
        float u = fmaf(Ps, inv_P_e, -1.0f);
        float e = expf(-u * u);
        M = alpha * u * u * e;
        Mp = 2.0f * alpha * inv_P_e * u * (1.0f - u * u) * e;
    }
};

__device__ __forceinline__ double mi64(double d, int per, double L)
{
    if (per) {
        double half = 0.5 * L;
        if (d > half) d -= L;
        else if (d < -half) d += L;
    }
    return d;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA sum of up to 4 per-thread values; thread 0 writes part[t * stride + blk] (FP64).
// Values are summed within a warp in their own type, then across warps in FP64 (every
// energy and load sum passes FP64 values: the mixed-precision kernels widen each atom's
// FP32 energy before any sum over atoms).
template <int NV, class T>
__device__ __forceinline__ void cta_partials(T (&v)[NV], double *part, int stride, int blk)
{
    __shared__ double sm[32][4];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int t = 0; t < NV; ++t) v[t] = warp_sum(v[t]);
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < NV; ++t) sm[wid][t] = (double)v[t];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            double acc = 0.0;
            for (int w = 0; w < nw; ++w) acc += sm[w][t];
            part[t * stride + blk] = acc;
        }
    }
}

// ============================================================================ Task 1 decision

// the position buffer of the state a step started from, and of the positions it evaluates
__device__ __forceinline__ int buf_cur(const DevArgs &a) { return (int)(*(volatile long long *)&a.st->ph_cur & 1); }
__device__ __forceinline__ int buf_step(const DevArgs &a) { return (int)(*(volatile long long *)&a.st->ph & 1); }

// Task 1 of a step (mode DEC_DRIFT, DEC_FULL or DEC_AUTO) or of an explicit list build
// (DEC_BUILD), and for a step also Task 2: the indenter moves by v dt, and the step count
// and the buffer counter advance (the pair kernels of this step find their positions in
// buffer ph & 1).  The graph's conditional h (use_cond) gets the rebuild decision; in
// DEC_AUTO, hv gets whether k_verlet1 runs (a rebuild, or no drift ready: drift_ok).
__global__ void k_decide(DevArgs a, int mode, int use_cond, cudaGraphConditionalHandle h, cudaGraphConditionalHandle hv)
{
    const int force = mode == DEC_BUILD;
    // the status words first, all at once (this kernel is a chain of dependent memory
    // accesses on the critical path of every step)
    const DevStatus *stc = a.st;
    const long long T = stc->ph;   // buffer counter of the state this step starts from
    const long long since = stc->since_build;
    const int drift_ok = stc->drift_ok, inner_next = stc->inner_ok_next;
    const unsigned imax_next = stc->imax_next;
    const int bs = (int)(T & 1);
    int any = 0;
    for (int r = threadIdx.x; r < a.n_rep; r += blockDim.x) {
        RepState &S = a.rs[r];
        const unsigned long long d0 = S.d2b[0], d1 = S.d2b[1];
        double dmax = sqrt(__longlong_as_double((long long)(bs ? d1 : d0)));
        S.d2b[bs] = 0ull;   // refilled by the force epilogue's drift to t + 2 dt
        int need;
        if (force) {
            need = 1;   // explicit build: no displacement test against a previous list
        } else if (a.rebuild_every > 0) {
            need = since >= a.rebuild_every;
            if (!need && 2.0 * dmax > a.skin) atomicOr(&a.st->err, MDE_SKIN);
        } else {
            need = (2.0 * dmax > a.skin) ||
                   (a.rep[r].n_c > 0 && __dadd_rn(dmax, fabs(__dsub_rn(S.z_ind, S.z_build))) > a.skin);
        }
        S.need = need;
        any |= need;
        S.z_cur = S.z_ind;
        if (!force) {
            // the rebuild tests of t + dt and t + 2 dt compare dmax with skin/2 and, with an
            // indenter in the displacement mode, with skin - |z_ind - z_build| as they will
            // be then (z_build = z_ind(t) if this step rebuilds).  A displacement below the
            // limit by more than the FP32 error of the estimate (< 1e-6 A) cannot change
            // that decision.
            const RepDev &Rr = a.rep[r];
            const double z1 = __dadd_rn(S.z_ind, __dmul_rn(Rr.v_ind, Rr.dt));
            const double z2 = __dadd_rn(z1, __dmul_rn(Rr.v_ind, Rr.dt));
            const double zb = need ? S.z_ind : S.z_build;
            double T1 = 0.5 * a.skin, T2 = 0.5 * a.skin;
            if (a.rebuild_every == 0 && Rr.n_c > 0) {
                T1 = fmin(T1, a.skin - fabs(z1 - zb));
                T2 = fmin(T2, a.skin - fabs(z2 - zb));
            }
            S.dthr = (float)(T1 - 1e-5);
            S.dthr2 = (float)(T2 - 1e-5);
            S.z_ind = z1;   // Task 2
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        const int run_verlet = mode == DEC_FULL || ((mode == DEC_DRIFT || mode == DEC_AUTO) && any) ||
                               (mode == DEC_AUTO && !drift_ok);
        if (mode == DEC_DRIFT && !any && !drift_ok) atomicOr(&a.st->err, MDE_SCHED);
        a.st->ph_cur = T;
        if (!force) { a.st->ph = T + 1; a.st->step += 1; }
        a.st->inner_ok = inner_next;   // a rebuild of the Verlet list below clears both
        a.st->imax_bits = run_verlet ? 0u : imax_next;
        a.st->imax_next = 0u;
        if (run_verlet)   // k_verlet1 fills the accumulator of the positions it makes
            for (int r = 0; r < a.n_rep; ++r) a.rs[r].d2b[bs ^ 1] = 0ull;
        a.st->any_rebuild = any;
        a.st->run_verlet = run_verlet;
        if (use_cond) {
            cudaGraphSetConditional(h, any ? 1u : 0u);
            if (mode == DEC_AUTO) cudaGraphSetConditional(hv, run_verlet ? 1u : 0u);
        }
    }
}
__global__ void k_zero_i32(int32_t *p, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = 0;
}

// wrap into the periodic box, FP64 cell coordinates, cell key, histogram
// Cell of every atom.  The exact result is cell_exact(wrap_exact(x)) in FP64.  When pos4
// holds the current positions (pos4_ok: k_verlet1 of the mixed path keeps it current,
// k_copyback writes it) the same result comes from the FP32 cell-relative position p
// about the old cell's centre: an atom farther than pad32 from every face of its old cell
// or of a face-adjacent cell is in that cell (pad32 bounds the w32 frame's drift from the
// FP64 grid plus the rounding of p), and a crossing of a periodic face moves x by exactly
// -+L, which is what wrap_exact computes there.  Every other atom (within pad32 of a face,
// moved by more than one cell, leaving a non-periodic domain, or not finite) takes the
// FP64 path.
__global__ void k_bin(DevArgs a)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) {
        // the list maxima describe the last build, unless an overflow is pending: then they
        // keep the largest count since, which the error message reports
        if (!(a.st->err & (MDE_OVERFLOW | MDE_COVERFLOW))) { a.st->max_cnt = 0; a.st->max_cntc = 0; }
        a.st->n_cand = 0; a.st->n_near = 0;
    }
    if (s >= a.S) return;
    int r = a.tile_rep[s / MD_TILE];
    const RepDev &R = a.rep[r];
    if (s - R.slot_off >= R.n_atoms) return;
    int c[3];
    bool done = false;
    const int b = buf_cur(a);
    double *x = a.xs[b];
    if (*(volatile int32_t *)&a.st->pos4_ok) {
        const int4 p = a.p4[b][s];
        const int pc = p.w;
        const float pr[3] = {qf(p.x, a.qu), qf(p.y, a.qu), qf(p.z, a.qu)};
        const int cc[3] = {cell_x(pc), cell_y(pc), cell_z(pc)};
        int wrap[3];
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float hw = 0.5f * R.w32[k], pad = R.pad32[k], q = pr[k];
            int d = 0;
            if (fabsf(q) < hw - pad) d = 0;
            else if (q > hw + pad && q < 3.0f * hw - pad) d = 1;
            else if (q < -hw - pad && q > pad - 3.0f * hw) d = -1;
            else ok = false;
            int cn = cc[k] + d;
            wrap[k] = 0;
            if (cn < 0 || cn >= R.nc[k]) {
                if (!R.per[k]) ok = false;
                wrap[k] = cn < 0 ? -1 : 1;
                cn -= wrap[k] * R.nc[k];
            }
            c[k] = cn;
        }
        if (ok) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (wrap[k]) {
                    const double xk = x[(size_t)k * a.S + s];
                    x[(size_t)k * a.S + s] = wrap[k] > 0 ? __dsub_rn(xk, R.L[k]) : __dadd_rn(xk, R.L[k]);
                }
            done = true;
        }
    }
    if (!done) {
        bool lost = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double xk = x[(size_t)k * a.S + s];
            if (xk != xk) lost = true;
            if (R.per[k]) {
                xk = wrap_exact(xk, R.lo[k], R.L[k], R.iL[k]);
                x[(size_t)k * a.S + s] = xk;
            } else if (xk < R.lo[k] || xk > R.hi[k]) {
                lost = true;
            }
            c[k] = cell_exact(xk, R.lo[k], R.w[k], R.iw[k], R.nc[k]);
        }
        if (lost) atomicOr(&a.st->err, MDE_LOST);
    }
    int key = R.cell_off + cell_key_loc(R, c[0], c[1], c[2]);
    a.key[s] = key;
    atomicAdd(&a.cell_count[key], 1);
}

__global__ void k_scan1(const int32_t *in, int32_t *out, int32_t *blk, int n)
{
    extern __shared__ int32_t sh[];
    int t = threadIdx.x, base = blockIdx.x * 2 * blockDim.x;
    int i0 = base + 2 * t, i1 = i0 + 1;
    int v0 = i0 < n ? in[i0] : 0, v1 = i1 < n ? in[i1] : 0;
    sh[t] = v0 + v1;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {   // Hillis-Steele inclusive scan of pair sums
        int add = t >= off ? sh[t - off] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    int excl = sh[t] - (v0 + v1);
    if (i0 < n) out[i0] = excl;
    if (i1 < n) out[i1] = excl + v0;
    if (t == blockDim.x - 1) blk[blockIdx.x] = sh[t];
}

// phase 2: one CTA scans the CTA totals (any count; chunks of blockDim)
__global__ void k_scan2(int32_t *blk, int nb)
{
    extern __shared__ int32_t sh[];
    int t = threadIdx.x;
    int carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + t;
        int v = i < nb ? blk[i] : 0;
        sh[t] = v;
        __syncthreads();
        for (int off = 1; off < (int)blockDim.x; off <<= 1) {
            int add = t >= off ? sh[t - off] : 0;
            __syncthreads();
            sh[t] += add;
            __syncthreads();
        }
        if (i < nb) blk[i] = carry + sh[t] - v;
        int tot = sh[blockDim.x - 1];
        __syncthreads();
        carry += tot;
    }
}

// phase 3: add CTA offsets and move each replica's cells to its TILE-aligned slot range
__global__ void k_scan3(DevArgs a, int per_block)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.total_cells) return;
    const RepDev &R = a.rep[a.cell_rep[c]];
    a.cell_start[c] += a.scan_blk[c / per_block] + (R.slot_off - R.real_off);
}

__global__ void k_scatter(DevArgs a)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const RepDev &R = a.rep[a.tile_rep[s / MD_TILE]];
    if (s - R.slot_off >= R.n_atoms) return;
    int key = a.key[s];
    int k = atomicAdd(&a.cell_fill[key], 1);
    a.perm[a.cell_start[key] + k] = s;
}

// deterministic order within a cell: ascending caller id (insertion sort, ~10 atoms)
// Atoms of a cell in ascending original index (one thread per cell, insertion sort), so
// the slot order and every list order are reproducible.  Skipped when an atom is lost (the
// step ends with MD_ERR_LOST_ATOM; non-finite positions all land in cell 0) and for a cell
// holding more than MD_SORT_MAX atoms (lists stay correct, their order is then the arrival
// order): neither case then costs quadratic time.
__global__ void k_cellsort(DevArgs a)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.total_cells) return;
    int b = a.cell_start[c], n = a.cell_count[c];
    if (n > MD_SORT_MAX || (*(volatile int32_t *)&a.st->err & MDE_LOST)) return;
    for (int i = 1; i < n; ++i) {
        int p = a.perm[b + i];
        int key = a.orig[p];
        int j = i - 1;
        while (j >= 0 && a.orig[a.perm[b + j]] > key) { a.perm[b + j + 1] = a.perm[b + j]; --j; }
        a.perm[b + j + 1] = p;
    }
}

__global__ void k_gather(DevArgs a)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const RepDev &R = a.rep[a.tile_rep[s / MD_TILE]];
    if (s - R.slot_off >= R.n_atoms) return;
    int o = a.perm[s];
    size_t S = a.S;
    const double *x = a.xs[buf_cur(a)];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.sx[k * S + s] = x[k * S + o];
        a.sv[k * S + s] = a.v[k * S + o];
        a.sF[k * S + s] = a.F[k * S + o];
    }
    a.sorig[s] = a.orig[o];
    a.sfixed[s] = a.fixed[o];
    int c0, c1, c2;
    key_cell_loc(R, a.key[o] - R.cell_off, c0, c1, c2);
    a.cellc[s] = pack_cell(c0, c1, c2);
}

// Fixed-point position of slot s about its cell centre lo + (c + 1/2) wc (see RepDev):
// round((x - centre) / u), u = 2^-k A.  x - centre is exact to ~1e-14 A in FP64 and the
// scaling by 2^k is exact, so the only rounding is to the unit (<= u/2).
__device__ __forceinline__ int4 rel_pos3(const DevArgs &a, const RepDev &R, int pc, double x0, double x1, double x2)
{
    const double c0 = __ldg(&a.cen[R.cen_off[0] + cell_x(pc)]);
    const double c1 = __ldg(&a.cen[R.cen_off[1] + cell_y(pc)]);
    const double c2 = __ldg(&a.cen[R.cen_off[2] + cell_z(pc)]);
    return make_int4(__double2int_rn((x0 - c0) * a.qinv), __double2int_rn((x1 - c1) * a.qinv),
                     __double2int_rn((x2 - c2) * a.qinv), pc);
}

__device__ __forceinline__ int4 rel_pos(const DevArgs &a, const RepDev &R, const double *x, int s)
{
    size_t S = a.S;
    return rel_pos3(a, R, a.cellc[s], x[s], x[S + s], x[2 * S + s]);
}

// position buffers: the state a step (or a list build) starts from, and the positions the
// pair kernels use (the state outside a step)

__global__ void k_copyback(DevArgs a)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const RepDev &R = a.rep[a.tile_rep[s / MD_TILE]];
    if (s - R.slot_off >= R.n_atoms) return;
    size_t S = a.S;
    const int b = buf_cur(a);
    double *x = a.xs[b];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double xk = a.sx[k * S + s];
        x[k * S + s] = xk;
        a.xb[k * S + s] = xk;
        a.v[k * S + s] = a.sv[k * S + s];
        a.F[k * S + s] = a.sF[k * S + s];
    }
    a.orig[s] = a.sorig[s];
    a.fixed[s] = a.sfixed[s];
    const int4 p = rel_pos(a, R, x, s);
    a.p4[b][s] = p;   // also used by the FP32 prefilter of k_nbr
    if (a.mixed) a.pb[s] = p;
    if (s == 0) a.st->pos4_ok = 1;
}

// full Cr-Cr Verlet list: every slot j != i in the 27-cell stencil with |x_j - x_i|^2 <
// (rc + skin)^2 decided in FP64.  A candidate whose FP32 distance (the exact fixed-point
// difference rounded once: error below 1e-6 relative with the unit rounding of both
// positions) is farther than 1e-5 (relative) from the cut-off is decided by that value;
// the rest take the exact FP64 test, so the set equals the all-FP64 set bit for bit.
//
// A lost atom (MDE_LOST from k_bin: outside a non-periodic domain or not finite) ends the
// step with MD_ERR_LOST_ATOM; the lists are then left empty rather than built around
// clamped atoms.  Otherwise every atom lies in its cell's box up to rounding, the box being
// off the w32-frame cell by at most pad32 (the frame's drift c |w - w32| plus 1e-4 A), so
// (i) a stencil cell whose widened box is farther than the cut-off from atom i holds no
// neighbour and is skipped, and (ii) every candidate is an in-cell atom.
__global__ void __launch_bounds__(128) k_nbr(DevArgs a)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const RepDev &R = a.rep[a.tile_rep[s / MD_TILE]];
    if (s - R.slot_off >= R.n_atoms) return;
    if (*(volatile int32_t *)&a.st->err & MDE_LOST) { a.cnt[s] = 0; return; }
    size_t S = a.S;
    const int bc = buf_cur(a);
    const double *x = a.xs[bc];
    const int4 *pos4 = a.p4[bc];
    const int4 pi = pos4[s];
    int pc = pi.w;
    int c0 = cell_x(pc), c1 = cell_y(pc), c2 = cell_z(pc);
    const float cut2 = (float)a.cut2;
    const float lo2 = cut2 * (1.0f - 1e-5f), hi2 = cut2 * (1.0f + 1e-5f);
    const float qu = a.qu;
    const float hx = fmaf(0.5f, R.w32[0], R.pad32[0]), hy = fmaf(0.5f, R.w32[1], R.pad32[1]),
                hz = fmaf(0.5f, R.w32[2], R.pad32[2]);
    int m = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int q2 = c2 + dz;
        if (q2 < 0 || q2 >= R.nc[2]) { if (!R.per[2]) continue; q2 = (q2 + R.nc[2]) % R.nc[2]; }
        // centre offset of the stencil cell in units: d Wq, plus d DLq through a periodic face
        const int tz = dz * R.Wq[2] + (c2 + dz != q2 ? dz * R.DLq[2] : 0) - pi.z;
        const float gz = fmaxf(fabsf(qf(tz, qu)) - hz, 0.0f);
        for (int dy = -1; dy <= 1; ++dy) {
            int q1 = c1 + dy;
            if (q1 < 0 || q1 >= R.nc[1]) { if (!R.per[1]) continue; q1 = (q1 + R.nc[1]) % R.nc[1]; }
            const int ty = dy * R.Wq[1] + (c1 + dy != q1 ? dy * R.DLq[1] : 0) - pi.y;
            const float gy = fmaxf(fabsf(qf(ty, qu)) - hy, 0.0f);
            const float gyz = fmaf(gy, gy, gz * gz);
            for (int dx = -1; dx <= 1; ++dx) {
                int q0 = c0 + dx;
                if (q0 < 0 || q0 >= R.nc[0]) { if (!R.per[0]) continue; q0 = (q0 + R.nc[0]) % R.nc[0]; }
                const int tx = dx * R.Wq[0] + (c0 + dx != q0 ? dx * R.DLq[0] : 0) - pi.x;
                const float gx = fmaxf(fabsf(qf(tx, qu)) - hx, 0.0f);
                if (fmaf(gx, gx, gyz) > hi2) continue;
                int key = R.cell_off + cell_key_loc(R, q0, q1, q2);
                int b = a.cell_start[key], e = b + a.cell_count[key];
                const unsigned dir = (dx < 0 ? 1u : 0u) | (dx > 0 ? 2u : 0u) | (dy < 0 ? 4u : 0u) | (dy > 0 ? 8u : 0u) |
                                     (dz < 0 ? 16u : 0u) | (dz > 0 ? 32u : 0u);
                for (int t0 = b; t0 < e; t0 += 4) {
                  // four candidate positions are loaded before any test or list store
                  int4 pjv[4];
#pragma unroll
                  for (int u = 0; u < 4; ++u) pjv[u] = __ldg(&pos4[min(t0 + u, e - 1)]);
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    const int t = t0 + u;
                    const bool valid = t < e && t != s;
                    const int4 pj = pjv[u];
                    const float fx = qf(pj.x + tx, qu), fy = qf(pj.y + ty, qu), fz = qf(pj.z + tz, qu);
                    const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                    bool in = r2f < lo2;
                    if (valid && !in && !(r2f > hi2)) {
                        double ddx = mi_exact(__dsub_rn(x[t], x[s]), R.per[0], R.L[0]);
                        double ddy = mi_exact(__dsub_rn(x[S + t], x[S + s]), R.per[1], R.L[1]);
                        double ddz = mi_exact(__dsub_rn(x[2 * S + t], x[2 * S + s]), R.per[2], R.L[2]);
                        in = norm2_exact(ddx, ddy, ddz) < a.cut2;
                    }
                    if (in && valid) {
                        if (m < a.kmax) a.nbr[(size_t)m * S + s] = (int32_t)((unsigned)t | (dir << MD_J_BITS));
                        ++m;
                    }
                  }
                }
            }
        }
    }
    a.cnt[s] = m < a.kmax ? m : a.kmax;
    if (m > a.kmax) atomicOr(&a.st->err, MDE_OVERFLOW);
    atomicMax(&a.st->max_cnt, m);
}

// Cr-C list through the indenter's own cell grid (indenter frame = positions at z_ind = 0),
// in two kernels.  k_nbrc: per atom, an FP32 rejection test against the grid's box; the
// few atoms it keeps (those under the indenter) are queued.  k_nbrc_near: one warp per
// queued atom, the lanes over the candidates of its cells, entries appended in candidate
// order (ballot), so the atoms under the indenter do not serialise in a few threads.
// Along a periodic axis both images of the film atom that can reach the indenter are
// searched: the cells of the two reach intervals are merged into one bit set per axis
// (indenter grids have at most 64 cells per axis), so every cell is visited once.
//
// The cells (bits) of an n-cell axis within reach r of offset u from the grid's origin
// (iw = 1 / cell width; r already widened by the caller's margin; bits a..b, b = 63 wraps
// to the top bit correctly)
__device__ __forceinline__ unsigned long long cell_bits32(float u, float r, float iw, int n)
{
    const float tl = floorf((u - r) * iw), th = floorf((u + r) * iw);
    if (!(th >= 0.0f) || !(tl <= (float)(n - 1))) return 0ull;
    const int a = tl < 0.0f ? 0 : (int)tl;
    const int b = th > (float)(n - 1) ? n - 1 : (int)th;
    return (2ull << b) - (1ull << a);
}

__global__ void __launch_bounds__(128) k_nbrc(DevArgs a)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    int r = a.tile_rep[s / MD_TILE];
    const RepDev &R = a.rep[r];
    if (s - R.slot_off >= R.n_atoms) return;
    a.cntc[s] = 0;
    if (R.n_c == 0 || (*(volatile int32_t *)&a.st->err & MDE_LOST)) return;
    // FP32 rejection: the atom's distance (minimum image) from the indenter grid's box
    // exceeds the reach on some axis.  x is rebuilt from the cell centre and the
    // cell-relative position with an error below 1e-4 A for coordinates below ~1e3 A;
    // the 0.01 A margin keeps every atom the exact test of k_nbrc_near could accept.
    // A non-finite position is queued (and then skipped: k_bin reports it).
    const int4 p = a.p4[buf_cur(a)][s];
    const int pc = p.w;
    const float pr[3] = {qf(p.x, a.qu), qf(p.y, a.qu), qf(p.z, a.qu)};
    const int cc[3] = {cell_x(pc), cell_y(pc), cell_z(pc)};
    const float zi32 = (float)a.rs[r].z_cur;
    const float lim = (float)a.cutc + 0.01f;
    bool far = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float d = fmaf((float)cc[k] + 0.5f, R.w32[k], R.lo32[k]) + pr[k] - (k == 2 ? zi32 : 0.0f) - R.cg_ctr32[k];
        if (R.per[k]) d = fmaf(-R.L32[k], rintf(d * R.iL32[k]), d);
        far |= fabsf(d) > R.cg_half32[k] + lim;
    }
    if (!far) a.cand[atomicAdd(&a.st->n_cand, 1)] = s;
}

__global__ void __launch_bounds__(256) k_nbrc_near(DevArgs a)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int n_cand = a.st->n_cand;
    const size_t S = a.S, C = a.C;
    const float cut2f = (float)a.cutc2, lo2 = cut2f * (1.0f - 1e-4f), hi2 = cut2f * (1.0f + 1e-4f);
    const double reach = a.cutc * (1.0 + 1e-9) + 1e-9;
    for (int qi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < n_cand; qi += nw) {
        const int s = a.cand[qi];
        const int r = a.tile_rep[s / MD_TILE];
        const RepDev &R = a.rep[r];
        const double z_ind = a.rs[r].z_cur;
        const double *x = a.xs[buf_cur(a)];
        const double xi[3] = {x[s], x[S + s], x[2 * S + s]};
        if (!(isfinite(xi[0]) && isfinite(xi[1]) && isfinite(xi[2]))) continue;   // reported by k_bin
        // the cells within reach along axis k = lane (lanes 0-2: the FP64 pipe of this part
        // takes a warp instruction whatever its active lanes, so once per axis), then
        // broadcast.  The image choice and the offsets from the grid's origin in FP64; the
        // cell range in FP32, widened by 0.01 A (FP32 errors here stay below 1e-4 A), so
        // that it holds every cell of the exact range: a wider range only adds candidates
        // the exact test rejects
        unsigned long long mk = 0ull;
        float qk = 0.0f;
        if (lane < 3) {
            const int k = lane;
            double q = (k == 0 ? xi[0] : k == 1 ? xi[1] : xi[2] - z_ind);
            const double ctr = R.cg_lo[k] + 0.5 * R.cg_n[k] * R.cg_w[k];
            const float rf = (float)reach + 0.01f, iwf = 1.0f / (float)R.cg_w[k];
            if (R.per[k]) {
                q = ctr + mi64(q - ctr, 1, R.L[k]);
                const double q2 = q > ctr ? q - R.L[k] : q + R.L[k];
                mk = cell_bits32((float)(q2 - R.cg_lo[k]), rf, iwf, R.cg_n[k]);
            }
            mk |= cell_bits32((float)(q - R.cg_lo[k]), rf, iwf, R.cg_n[k]);
            qk = (float)(q - R.cg_lo[k]);
        }
        unsigned long long mask[3];
        float q32[3];
        bool none = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mask[k] = __shfl_sync(0xffffffffu, mk, k);
            q32[k] = __shfl_sync(0xffffffffu, qk, k);
            none |= !mask[k];
        }
        if (none) continue;
        // FP32 prefilter (indenter frame, positions below ~100 A: error < 1e-4 A^2 on y^2);
        // the exact FP64 test decides every candidate within 1e-4 (relative) of the cut-off
        int m = 0;
        for (unsigned long long m2 = mask[2]; m2; m2 &= m2 - 1) {
            const int q2 = __ffsll((long long)m2) - 1;
            for (unsigned long long m1 = mask[1]; m1; m1 &= m1 - 1) {
                const int q1 = __ffsll((long long)m1) - 1;
                for (unsigned long long m0 = mask[0]; m0; m0 &= m0 - 1) {
                    const int q0 = __ffsll((long long)m0) - 1;
                    const int key = R.ccell_off + (q2 * R.cg_n[1] + q1) * R.cg_n[0] + q0;
                    const int b = a.ccell_start[key], e = b + a.ccell_count[key];
                    for (int c0 = b; c0 < e; c0 += 32) {
                        const int c = c0 + lane;
                        bool in = false;
                        if (c < e) {
                            const float4 pc = __ldg(&a.xc32[c]);
                            float fx = pc.x - q32[0], fy = pc.y - q32[1], fz = pc.z - q32[2];
                            if (R.per[0]) fx = fmaf(-R.L32[0], rintf(fx * R.iL32[0]), fx);
                            if (R.per[1]) fy = fmaf(-R.L32[1], rintf(fy * R.iL32[1]), fy);
                            if (R.per[2]) fz = fmaf(-R.L32[2], rintf(fz * R.iL32[2]), fz);
                            const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                            in = r2f < lo2;
                            if (!in && !(r2f > hi2)) {
                                double ddx = mi_exact(__dsub_rn(a.xc0[c], xi[0]), R.per[0], R.L[0]);
                                double ddy = mi_exact(__dsub_rn(a.xc0[C + c], xi[1]), R.per[1], R.L[1]);
                                double zc = __dadd_rn(a.xc0[2 * C + c], z_ind);
                                double ddz = mi_exact(__dsub_rn(zc, xi[2]), R.per[2], R.L[2]);
                                in = norm2_exact(ddx, ddy, ddz) < a.cutc2;
                            }
                        }
                        const unsigned bal = __ballot_sync(0xffffffffu, in);
                        if (in) {
                            const int pos = m + __popc(bal & ((1u << lane) - 1u));
                            if (pos < a.kcmax) a.nbrc[(size_t)pos * S + s] = c;
                        }
                        m += __popc(bal);
                    }
                }
            }
        }
        if (lane == 0) {
            a.cntc[s] = m < a.kcmax ? m : a.kcmax;
            if (m > a.kcmax) atomicOr(&a.st->err, MDE_COVERFLOW);
            atomicMax(&a.st->max_cntc, m);
            if (m > 0) a.near[atomicAdd(&a.st->n_near, 1)] = s;
        }
    }
}

__global__ void k_build_done(DevArgs a)
{
    for (int r = threadIdx.x; r < a.n_rep; r += blockDim.x) a.rs[r].z_build = a.rs[r].z_cur;
    if (threadIdx.x == 0) {
        a.st->rebuilds += 1; a.st->since_build = 0;
        a.st->inner_ok = 0; a.st->inner_ok_next = 0;   // slots were permuted: the inner list is stale
        a.st->drift_ok = 0;                             // and so is a drift made before the rebuild
    }
}

// ============================================================================ list check

// The debug check of the lists of the last build (no counterpart in the paper: it stands
// in for a memory checker, by testing every invariant the pair kernels rely on when they
// index memory with list entries).  One thread per atom, counts by kind into st->chk:
//   0 an entry outside the atom's replica or naming the atom itself, 1 a length above the
//   capacity, 2 a direction code that does not match the two atoms' cells, 3 a listed pair
//   at or beyond `radius` at the build positions (exact FP64), 4 a pair within `radius`
//   there that is missing, 5 a pair listed one way only, 6 a Cr-C entry outside the
//   replica's indenter or beyond rc_m + skin at the build, 7 an inner-list entry that is
//   not in the Verlet list (checked when the inner list belongs to the current build).
// Any violation also raises MDE_LISTCHECK.
__global__ void __launch_bounds__(128) k_check_lists(DevArgs a, double radius)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const RepDev &R = a.rep[a.tile_rep[s / MD_TILE]];
    if (s - R.slot_off >= R.n_atoms) return;
    const size_t S = a.S;
    const double r2max = radius * radius;
    unsigned long long bad[MD_NCHK] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int n = a.cnt[s];
    if (n < 0 || n > a.kmax) bad[1]++;
    const int m = min(max(n, 0), a.kmax);
    const int ci = a.cellc[s];
    const int cc[3] = {cell_x(ci), cell_y(ci), cell_z(ci)};
    auto dist2 = [&](int j) {
        const double dx = mi_exact(__dsub_rn(a.xb[j], a.xb[s]), R.per[0], R.L[0]);
        const double dy = mi_exact(__dsub_rn(a.xb[S + j], a.xb[S + s]), R.per[1], R.L[1]);
        const double dz = mi_exact(__dsub_rn(a.xb[2 * S + j], a.xb[2 * S + s]), R.per[2], R.L[2]);
        return norm2_exact(dx, dy, dz);
    };
    auto listed = [&](int i, unsigned j) {   // j (low bits) in the Verlet row of i
        const int ni = min(max(a.cnt[i], 0), a.kmax);
        for (int k = 0; k < ni; ++k)
            if (((unsigned)a.nbr[(size_t)k * S + i] & MD_J_MASK) == j) return true;
        return false;
    };
    for (int k = 0; k < m; ++k) {
        const unsigned e = (unsigned)a.nbr[(size_t)k * S + s];
        const int j = (int)(e & MD_J_MASK);
        if (j < R.slot_off || j - R.slot_off >= R.n_atoms || j == s) { bad[0]++; continue; }
        const int cj = a.cellc[j];
        const int dj[3] = {cell_x(cj) - cc[0], cell_y(cj) - cc[1], cell_z(cj) - cc[2]};
        unsigned dir = 0u;
        bool ok = true;
        for (int q = 0; q < 3; ++q) {
            int d = dj[q];
            if (R.per[q] && d > 1) d -= R.nc[q];
            if (R.per[q] && d < -1) d += R.nc[q];
            if (d < -1 || d > 1) ok = false;
            dir |= (d < 0 ? 1u : 0u) << (2 * q);
            dir |= (d > 0 ? 2u : 0u) << (2 * q);
        }
        if (!ok || dir != (e >> MD_J_BITS)) bad[2]++;
        if (!(dist2(j) < r2max)) bad[3]++;
        if (!listed(j, (unsigned)s)) bad[5]++;
    }
    // completeness: every atom of the stencil cells within radius of s at the build
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int q[3] = {cc[0] + dx, cc[1] + dy, cc[2] + dz};
                bool skip = false;
                for (int t = 0; t < 3; ++t) {
                    if (q[t] < 0 || q[t] >= R.nc[t]) {
                        if (!R.per[t]) skip = true;
                        q[t] = (q[t] + R.nc[t]) % R.nc[t];
                    }
                }
                if (skip) continue;   // (a periodic axis has >= 3 cells: no cell is visited twice)
                const int key = R.cell_off + cell_key_loc(R, q[0], q[1], q[2]);
                const int b = a.cell_start[key], e = b + a.cell_count[key];
                for (int t = b; t < e; ++t)
                    if (t != s && dist2(t) < r2max && !listed(s, (unsigned)t)) bad[4]++;
            }
    // Cr-C list, at the indenter's displacement of the build
    const int nc = a.cntc[s];
    if (nc < 0 || nc > a.kcmax) bad[1]++;
    const double zb = a.rs[a.tile_rep[s / MD_TILE]].z_build;
    for (int k = 0; k < min(max(nc, 0), a.kcmax); ++k) {
        const int c = a.nbrc[(size_t)k * S + s];
        if (c < R.c_off || c - R.c_off >= R.n_c) { bad[6]++; continue; }
        const size_t C = a.C;
        const double dx = mi_exact(__dsub_rn(a.xc0[c], a.xb[s]), R.per[0], R.L[0]);
        const double dy = mi_exact(__dsub_rn(a.xc0[C + c], a.xb[S + s]), R.per[1], R.L[1]);
        const double dz = mi_exact(__dsub_rn(__dadd_rn(a.xc0[2 * C + c], zb), a.xb[2 * S + s]), R.per[2], R.L[2]);
        if (!(norm2_exact(dx, dy, dz) < a.cutc2)) bad[6]++;
    }
    // inner list (mixed precision), when it belongs to this build
    if (a.mixed && (a.st->inner_ok || a.st->inner_ok_next)) {
        const int ni = a.icnt[s];
        if (ni < 0 || ni > a.kinner) bad[1]++;
        for (int k = 0; k < min(max(ni, 0), a.kinner); ++k) {
            const unsigned e = (unsigned)a.inner[(size_t)k * S + s];
            if ((e & MD_J_MASK) == (unsigned)s) continue;   // padding of a lane group
            bool found = false;
            for (int kk = 0; kk < m && !found; ++kk) found = (unsigned)a.nbr[(size_t)kk * S + s] == e;
            if (!found) bad[7]++;
        }
    }
    bool any = false;
    for (int t = 0; t < MD_NCHK; ++t)
        if (bad[t]) { atomicAdd(&a.st->chk[t], bad[t]); any = true; }
    if (any) atomicOr(&a.st->err, MDE_LISTCHECK);
}

__global__ void k_zero_chk(DevArgs a)
{
    if (threadIdx.x < MD_NCHK) a.st->chk[threadIdx.x] = 0ull;
}

// ============================================================================ Tasks 2 + 3

// Task 3 of one atom (Eqs. A11-A12: half kick, drift) from its state (x, v, F) at time t:
// v(t + dt/2) to vh, x(t + dt) and its cell-relative copy to the buffers xd, pd, and the
// displacement tests of x(t + dt): since the Verlet-list build (d2bits, for the rebuild
// test; FP32 estimate from the cell-relative positions when it is below thr by more than
// its error, else exact FP64) and, in mixed precision, since the inner-list build (ibits).
// Fixed atoms keep x and v (they are copied).  pc: the atom's cell at the last list build.
__device__ __forceinline__ void drift_atom(const DevArgs &a, const RepDev &R, int s, int pc, float thr,
                                           double x0, double x1, double x2, double v0, double v1, double v2,
                                           double F0, double F1, double F2, double *xd, int4 *pd,
                                           unsigned long long &d2bits, unsigned &ibits)
{
    const size_t S = a.S;
    if (!a.fixed[s]) {
        const double hk = R.hk;
        v0 = fma(hk, F0, v0); v1 = fma(hk, F1, v1); v2 = fma(hk, F2, v2);                 // Eq. A12
        x0 = fma(R.dt, v0, x0); x1 = fma(R.dt, v1, x1); x2 = fma(R.dt, v2, x2);           // Eq. A11
    }
    a.vh[s] = v0; a.vh[S + s] = v1; a.vh[2 * S + s] = v2;
    xd[s] = x0; xd[S + s] = x1; xd[2 * S + s] = x2;
    bool exact = true;
    if (a.mixed) {
        const int4 p = rel_pos3(a, R, pc, x0, x1, x2);
        pd[s] = p;
        // same cell frame as the build's copy pb: a displacement clearly below thr cannot
        // change the rebuild test and its exact FP64 value is not needed
        const int4 b = a.pb[s];
        const float bx = qf(p.x - b.x, a.qu), by = qf(p.y - b.y, a.qu), bz = qf(p.z - b.z, a.qu);
        const float d2f = fmaf(bx, bx, fmaf(by, by, bz * bz));
        exact = !(thr > 0.0f && d2f < thr * thr);
        // displacement since the inner list was rebuilt (same cell frame: a rebuild of the
        // Verlet list in between invalidates the inner list anyway)
        const int4 q = a.pin[s];
        const float ex = qf(p.x - q.x, a.qu), ey = qf(p.y - q.y, a.qu), ez = qf(p.z - q.z, a.qu);
        float dm2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        if (!(dm2 <= 1e30f)) dm2 = 1e30f;   // not finite: force the rebuild
        ibits = __float_as_uint(dm2);       // dm2 >= 0: bit order = value order
    }
    if (exact) {
        double d2 = norm2_exact(__dsub_rn(x0, a.xb[s]), __dsub_rn(x1, a.xb[S + s]), __dsub_rn(x2, a.xb[2 * S + s]));
        if (d2 != d2) d2 = 1e300;   // NaN position: force a rebuild, which reports it
        d2bits = (unsigned long long)__double_as_longlong(d2);   // d2 >= 0: bit order = value order
    }
}

// maxima of a CTA's d2bits and ibits into *d2max and *imax (every thread of the CTA calls it)
__device__ __forceinline__ void cta_max_disp(unsigned long long d2bits, unsigned ibits,
                                             unsigned long long *d2max, unsigned *imax)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, d2bits, o);
        d2bits = t > d2bits ? t : d2bits;
        ibits = max(ibits, __shfl_xor_sync(0xffffffffu, ibits, o));
    }
    __shared__ unsigned long long sm[32];
    __shared__ unsigned smi[32];
    const int nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) { sm[threadIdx.x >> 5] = d2bits; smi[threadIdx.x >> 5] = ibits; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0ull;
        unsigned mi = 0u;
        for (int w = 0; w < nw; ++w) { m = sm[w] > m ? sm[w] : m; mi = max(mi, smi[w]); }
        if (m) atomicMax(d2max, m);
        if (mi) atomicMax(imax, mi);
    }
}

// Task 3 when the last step's force epilogue did not make it (first step after a state was
// set, or a rebuild this step): from the state in buffer ph_cur & 1 to buffer ph & 1 (one
// buffer in FP64 mode: in place).  One CTA = one tile (one replica).
__global__ void __launch_bounds__(MD_TILE) k_verlet1(DevArgs a)
{
    const int s = blockIdx.x * MD_TILE + threadIdx.x;
    const int r = a.tile_rep[blockIdx.x];
    const RepDev &R = a.rep[r];
    if (s == 0 && !a.mixed) a.st->pos4_ok = 0;   // the FP64 path does not keep pos4 current
    const int bs = buf_cur(a), bd = buf_step(a);
    unsigned long long d2bits = 0ull;
    unsigned ibits = 0u;
    if (s - R.slot_off < R.n_atoms) {
        const size_t S = a.S;
        const double *x = a.xs[bs];
        drift_atom(a, R, s, a.cellc[s], a.rs[r].dthr, x[s], x[S + s], x[2 * S + s], a.v[s], a.v[S + s], a.v[2 * S + s],
                   a.F[s], a.F[S + s], a.F[2 * S + s], a.xs[bd], a.p4[bd], d2bits, ibits);
    }
    cta_max_disp(d2bits, ibits, &a.rs[r].d2b[bd], &a.st->imax_bits);
}

// Before a force pass that drifts a state set from outside (integrate = 2): per replica
// the threshold below which the displacement of the drifted positions cannot decide the
// rebuild test that examines them (as k_decide sets it when it advances a step, with the
// lists of the last build), and the accumulators of that test and of the inner list's
// test cleared.
__global__ void k_drift_prep(DevArgs a)
{
    const int b = (int)((a.st->ph + 1) & 1);
    for (int r = threadIdx.x; r < a.n_rep; r += blockDim.x) {
        RepState &S = a.rs[r];
        const RepDev &Rr = a.rep[r];
        double T1 = 0.5 * a.skin;
        if (a.rebuild_every == 0 && Rr.n_c > 0) {
            const double z1 = __dadd_rn(S.z_ind, __dmul_rn(Rr.v_ind, Rr.dt));
            T1 = fmin(T1, a.skin - fabs(z1 - S.z_build));
        }
        S.dthr = (float)(T1 - 1e-5);
        S.d2b[b] = 0ull;
    }
    if (threadIdx.x == 0) a.st->imax_next = 0u;
}

// md_set_state, before the new positions: the error word cleared, replica r's indenter
// displacement and the step count set, its accumulator for the rebuild test of the state
// positions zeroed, the drift made from the old state voided.  The inner list's
// displacement max keeps the other replicas' current values (their positions do not
// change) unless the last k_density rebuilt that list, which makes them all 0.
__global__ void k_state_prep(DevArgs a, int r, double z_ind, long long step)
{
    if (threadIdx.x != 0) return;
    DevStatus *st = a.st;
    st->err = 0;
    st->step = step;
    st->drift_ok = 0;
    st->inner_ok = st->inner_ok_next;
    if (st->imax_fresh) st->imax_bits = 0u;
    st->pos4_ok = a.mixed;   // FP64: the other replicas' pos4 are not kept current
    RepState &S = a.rs[r];
    st->changed = S.z_ind != z_ind;   // k_state_scan adds the positions
    S.z_ind = z_ind;
    S.d2b[st->ph & 1] = 0ull;
}

// md_set_state for the n atoms of replica r (slots slot_off ...): the new positions (from
// stage in caller order, or the current ones when stage is NULL) into the state buffer,
// noting whether any differs from the one it replaces,
// their pos4, the exact FP64 max |x - x_build|^2 (as the drift reduces it for k_decide)
// and, in mixed precision, the displacement since the inner list was built.
__global__ void __launch_bounds__(256) k_state_scan(DevArgs a, int r, int slot_off, int n, const double *stage)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const RepDev &R = a.rep[r];
    const int b = buf_step(a);
    unsigned long long d2bits = 0ull;
    unsigned ibits = 0u;
    if (i < n) {
        const size_t S = a.S;
        const int s = slot_off + i;
        double *x = a.xs[b];
        double x0, x1, x2;
        if (stage) {
            const int o = a.orig[s];
            x0 = stage[3 * (size_t)o]; x1 = stage[3 * (size_t)o + 1]; x2 = stage[3 * (size_t)o + 2];
            // bitwise comparison (a NaN counts as changed)
            if (!(x0 == x[s] && x1 == x[S + s] && x2 == x[2 * S + s])) a.st->changed = 1;
            x[s] = x0; x[S + s] = x1; x[2 * S + s] = x2;
        } else {
            x0 = x[s]; x1 = x[S + s]; x2 = x[2 * S + s];
        }
        const int4 p = rel_pos3(a, R, a.cellc[s], x0, x1, x2);
        a.p4[b][s] = p;
        double d2 = norm2_exact(__dsub_rn(x0, a.xb[s]), __dsub_rn(x1, a.xb[S + s]), __dsub_rn(x2, a.xb[2 * S + s]));
        if (d2 != d2) d2 = 1e300;   // NaN position: force a rebuild, which reports it
        d2bits = (unsigned long long)__double_as_longlong(d2);
        if (a.mixed) {
            const int4 q = a.pin[s];
            const float ex = qf(p.x - q.x, a.qu), ey = qf(p.y - q.y, a.qu), ez = qf(p.z - q.z, a.qu);
            float dm2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (!(dm2 <= 1e30f)) dm2 = 1e30f;
            ibits = __float_as_uint(dm2);
        }
    }
    cta_max_disp(d2bits, ibits, &a.rs[r].d2b[b], &a.st->imax_bits);
}

// the displacement rule of k_decide on every replica's state positions (whatever the
// rebuild mode: the caller's positions are not integrator steps), into any_rebuild
__global__ void k_state_need(DevArgs a)
{
    const int b = buf_step(a);
    int any = 0;
    for (int r = threadIdx.x; r < a.n_rep; r += blockDim.x) {
        const RepState &S = a.rs[r];
        const double dmax = sqrt(__longlong_as_double((long long)S.d2b[b]));
        any |= (2.0 * dmax > a.skin) ||
               (a.rep[r].n_c > 0 && __dadd_rn(dmax, fabs(__dsub_rn(S.z_ind, S.z_build))) > a.skin);
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) a.st->any_rebuild = any;
}

// ============================================================================ Task 4, mixed precision
//
// Geometry of a pair from fixed-point cell-relative positions: x_j - x_i = (p_j - p_i) +
// offset, in units u, the offset being the centre-to-centre vector of the two cells, read
// from a 64-entry table indexed by the direction bits of the list entry (multiples of Wq);
// a pair that crosses a periodic face (atom i in an edge cell, direction bit towards that
// face) adds -+DLq on that axis.  The integer sum is exact; converted to FP32 (and scaled
// by u, a power of two) it is the displacement rounded once.  Positions in FP32 about the
// cell centres would carry three roundings (both positions and the sum), three times the
// error, and the FP32 pair forces would then miss 1e-5 relative on cold or perfect
// lattices, where the net forces are small.

struct PairGeom {
    unsigned xmask;          // direction bits that cross a periodic face for this atom
    int dL0, dL1, dL2;
};

__device__ __forceinline__ void fill_offsets(int4 *sm_off, const RepDev &R)
{
    for (int c = threadIdx.x; c < 64; c += blockDim.x) {
        int ox = (c & 1 ? -R.Wq[0] : 0) + (c & 2 ? R.Wq[0] : 0);
        int oy = (c & 4 ? -R.Wq[1] : 0) + (c & 8 ? R.Wq[1] : 0);
        int oz = (c & 16 ? -R.Wq[2] : 0) + (c & 32 ? R.Wq[2] : 0);
        sm_off[c] = make_int4(ox, oy, oz, 0);
    }
}

__device__ __forceinline__ PairGeom pair_geom(const RepDev &R, int ci)
{
    PairGeom G;
    const int c0 = cell_x(ci), c1 = cell_y(ci), c2 = cell_z(ci);
    G.xmask = (R.per[0] && c0 == 0 ? 1u : 0u) | (R.per[0] && c0 == R.nc[0] - 1 ? 2u : 0u) |
              (R.per[1] && c1 == 0 ? 4u : 0u) | (R.per[1] && c1 == R.nc[1] - 1 ? 8u : 0u) |
              (R.per[2] && c2 == 0 ? 16u : 0u) | (R.per[2] && c2 == R.nc[2] - 1 ? 32u : 0u);
    G.dL0 = R.DLq[0]; G.dL1 = R.DLq[1]; G.dL2 = R.DLq[2];
    return G;
}

// PER = false: no atom of the warp sits in an edge cell of a periodic axis, so no pair
// crosses a periodic face and the correction is left out (the caller decides per warp, so
// the branch between the two forms is uniform)
// The displacement is returned in units of qu (FP32, one rounding): the callers scale r^2
// by qu^2 and a force sum by qu once (exact powers of two, so every result is bit for bit
// what the same arithmetic on displacements in A gives).
template <bool PER>
__device__ __forceinline__ void disp(const int4 &pi, const int4 &pj, unsigned dir, const int4 *sm_off,
                                     const PairGeom &G, float &dx, float &dy, float &dz)
{
    const int4 o = sm_off[dir];
    int ix = pj.x - pi.x + o.x, iy = pj.y - pi.y + o.y, iz = pj.z - pi.z + o.z;
    if (PER) {
        const unsigned c = dir & G.xmask;
        if (c) {   // through a periodic face: the period is nc Wq + DLq
            ix += (c & 1 ? -G.dL0 : 0) + (c & 2 ? G.dL0 : 0);
            iy += (c & 4 ? -G.dL1 : 0) + (c & 8 ? G.dL1 : 0);
            iz += (c & 16 ? -G.dL2 : 0) + (c & 32 ? G.dL2 : 0);
        }
    }
    dx = __int2float_rn(ix); dy = __int2float_rn(iy); dz = __int2float_rn(iz);
}

template <bool B> struct BoolC { static constexpr bool value = B; };

// A list entry is read once: loaded around L1 (no allocation there), so the rows do not
// evict the neighbour positions the gathers reuse (~1 % of a step)
__device__ __forceinline__ unsigned ld_stream(const int32_t *p)
{
    unsigned v;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16); no registers, no wait
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The pair loops of the mixed path evaluate the forms of Eqs. A2 and A4 directly in FP32
// (no table gather: at FP32 resolution a Hermite table adds nothing but 32 bytes of memory
// traffic per pair; its deviation from the forms is below 1e-11).  f: for an even integer
// beta the power (f_e^(2/beta) r_e^2 / r^2)^(beta/2) by multiplication; Phi: about t = tc
// (PotF32).  IPOW > 0: beta = 2 IPOW known at compile time; IPOW = 0: from Q.ipow, else
// the exp2/log2 form.
template <int IPOW>
__device__ __forceinline__ float f_pow(const Pot32 &Q, float q, float r)
{
    if (IPOW > 0 || Q.ipow > 0) {
        float fr = q;
        if (IPOW > 0) {
#pragma unroll
            for (int k = 1; k < IPOW; ++k) fr *= q;
        } else {
            for (int k = 1; k < Q.ipow; ++k) fr *= q;
        }
        return fr;
    }
    return exp2f(Q.lf0 - Q.beta * log2f(r));
}

// 1/sqrt(r2) refined by a Newton step
__device__ __forceinline__ float rsqrt_nr(float r2)
{
    const float y = rsqrtf(r2);
    return y * fmaf(-0.5f * r2 * y, y, 1.5f);
}

// f(r) of the density pass.  q = re2f / r^2 from one reciprocal refined by a Newton step
// (about 1 ulp: the densities' rounding feeds F'(rho) of every neighbour); r itself enters
// only the shifted-force term r f'(rc) (f'(rc) is ~4 % of f' at the first shell), where the
// unrefined square root's 2 ulp are negligible -- except in the exp2/log2 form of f.
template <int IPOW>
__device__ __forceinline__ float fa_val(const Pot32 &Q, float r2)
{
    const bool gen = IPOW == 0 && Q.ipow == 0;
    const float r = r2 * (gen ? rsqrt_nr(r2) : rsqrtf(r2));
    const float rcp = __fdividef(1.0f, r2);
    float q = Q.re2f * rcp;
    q = fmaf(rcp, fmaf(-q, r2, Q.re2f), q);
    return fmaf(-r, Q.df_rc, f_pow<IPOW>(Q, q, r) - Q.cf);
}

// f, f' and Phi' of a pair (force pass), and Phi itself when EN (the energies are wanted),
// from r2 and the refined 1/r (the force's direction factor): r = r2 / r, q = re2f / r^2.
// Phi beyond its double root (t > 0) is zero with its slope; t is clamped to 0 there, where
// both forms (t^2 times a cubic in s, t times a cubic in s) give exactly 0.
template <int IPOW, bool EN>
__device__ __forceinline__ void fa_phi(const Pot32 &Q, float r2, float rinv, float &f, float &df, float &ph, float &dph)
{
    const float r = r2 * rinv;
    const float fr = f_pow<IPOW>(Q, Q.re2f * (rinv * rinv), r);
    f = fmaf(-r, Q.df_rc, fr - Q.cf);
    const float beta = IPOW > 0 ? 2.0f * IPOW : Q.beta;
    df = fmaf(-beta * fr, rinv, -Q.df_rc);
    const float sv = (r - Q.rs) * Q.inv_re;   // t - tc
    const float t = fminf(sv + Q.tc, 0.0f);
    ph = EN ? t * t * fmaf(fmaf(fmaf(Q.b3, sv, Q.b2), sv, Q.b1), sv, Q.b0) : 0.0f;
    dph = t * fmaf(fmaf(fmaf(Q.c3, sv, Q.c2), sv, Q.c1), sv, Q.c0);
}

// The force pass's pair terms for beta = 6 (f = q^3, q = re2f / r^2) for two pairs at once,
// in Blackwell's packed FP32x2 arithmetic (__ffma2_rn, __fmul2_rn, __fadd2_rn: each
// component rounded as the scalar operation; the rsqrt and Phi's clamp per component), as
// an explicit sequence of separately rounded operations.  In: the two displacements in
// units of qu and (F'_j, 2 M'_j); out: r^2, coef (the force on i from j over its
// displacement) and, with EN, Phi/2; the caller selects coef and Phi/2 by r < rc.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

template <bool EN>
__device__ __forceinline__ void pair_force6x2(const Pot32 &Q, float qu2, float2 fmi, float2 fmj0, float2 fmj1,
                                              float2 DX, float2 DY, float2 DZ, float2 &R2, float2 &COEF,
                                              float2 &PH)
{
    R2 = __fmul2_rn(__ffma2_rn(DX, DX, __ffma2_rn(DY, DY, __fmul2_rn(DZ, DZ))), f2(qu2));
    const float2 Y = make_float2(rsqrtf(R2.x), rsqrtf(R2.y));
    const float2 RINV = __fmul2_rn(Y, __ffma2_rn(__fmul2_rn(__fmul2_rn(R2, f2(-0.5f)), Y), Y, f2(1.5f)));
    const float2 R = __fmul2_rn(R2, RINV);
    const float2 QQ = __fmul2_rn(f2(Q.re2f), __fmul2_rn(RINV, RINV));
    const float2 FR = __fmul2_rn(__fmul2_rn(QQ, QQ), QQ);
    const float2 F = __ffma2_rn(R, f2(-Q.df_rc), __fadd2_rn(FR, f2(-Q.cf)));
    const float2 DF = __ffma2_rn(__fmul2_rn(FR, f2(-6.0f)), RINV, f2(-Q.df_rc));
    const float2 SV = __fmul2_rn(__fadd2_rn(R, f2(-Q.rs)), f2(Q.inv_re));
    float2 T = __fadd2_rn(SV, f2(Q.tc));
    T.x = fminf(T.x, 0.0f);
    T.y = fminf(T.y, 0.0f);
    const float2 PC = __ffma2_rn(__ffma2_rn(__ffma2_rn(f2(Q.c3), SV, f2(Q.c2)), SV, f2(Q.c1)), SV, f2(Q.c0));
    const float2 DPH = __fmul2_rn(T, PC);
    const float2 A = __fadd2_rn(f2(fmi.y), make_float2(fmj0.y, fmj1.y));
    const float2 B = __fadd2_rn(f2(fmi.x), make_float2(fmj0.x, fmj1.x));
    COEF = __fmul2_rn(__ffma2_rn(__ffma2_rn(A, F, B), DF, DPH), RINV);
    if (EN) {
        const float2 PB = __ffma2_rn(__ffma2_rn(__ffma2_rn(f2(Q.b3), SV, f2(Q.b2)), SV, f2(Q.b1)), SV, f2(Q.b0));
        PH = __fmul2_rn(__fmul2_rn(__fmul2_rn(T, T), PB), f2(0.5f));
    } else {
        PH = make_float2(0.0f, 0.0f);
    }
}

// Task 4a (Eqs. A2-A3): rho_i, P_i over the pairs within rc; F'(rho_i), M'(P_i) stored,
// and with EN F(rho_i), M(P_i) into the CTA's energy partials.  MD_UNROLL entries per lane
// are loaded (list entry, then position) before any is used.
//
// The inner list (Sec. 2.6) holds the Verlet-list entries within rc + inner skin at its
// last rebuild, in Verlet-list order.  Every pair within rc is in it while no atom has
// moved more than half the skin since (k_verlet1 reduces the displacement); then this
// kernel rebuilds it from the Verlet list.  With inner skin < 0 it is rebuilt every step
// with radius rc, as in the paper.  Both loops take the pairs within rc in Verlet-list
// order, so the sums do not depend on which list a step uses.
// The launch bound caps the kernel at 51 registers: with both loops in one kernel the
// compiler otherwise takes 60-64 and the loss of occupancy costs ~10 %.
template <int TPA, int IPOW, bool EN>
__global__ void __launch_bounds__(256, 5) k_density_mixed(DevArgs a, PotDev P)
{
    __shared__ int4 sm_off[64];
    const int A = blockDim.x / TPA;
    const int g = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int s = blockIdx.x * A + g;
    const RepDev &R = a.rep[a.tile_rep[(blockIdx.x * A) / MD_TILE]];
    fill_offsets(sm_off, R);
    __syncthreads();
    const Pot32 &Q = static_cast<const Pot32 &>(P.q);
    const bool real = (s - R.slot_off) < R.n_atoms;
    const size_t S = a.S;
    // uniform over the launch: nothing below writes inner_ok or imax_bits
    const bool rebuild = !a.st->inner_ok || !(__uint_as_float(a.st->imax_bits) <= a.ithr2);
    float rho = 0.f, Ps = 0.f;
    int m = 0;   // inner-list entries of this lane
    const int4 *pp = a.p4[buf_step(a)];   // positions x(t + dt)
    const int4 pi = pp[s];
    const PairGeom G = pair_geom(R, pi.w);
    const float qu2 = a.qu * a.qu;   // r^2 from displacements in units of qu
    const bool per = __any_sync(0xffffffffu, real && G.xmask != 0u);
    auto work = [&](auto PERC) {
        constexpr bool PER = decltype(PERC)::value;
        if (!real) return;
        if (rebuild) {
            const int n = a.cnt[s];
            for (int k0 = lane; k0 < n; k0 += TPA * MD_UNROLL) {
                unsigned e[MD_UNROLL];
#pragma unroll
                for (int u = 0; u < MD_UNROLL; ++u) {
                    const int k = k0 + u * TPA;
                    e[u] = k < n ? (unsigned)__ldg(&a.nbr[(size_t)k * S + s]) : (unsigned)s;
                }
                int4 pj[MD_UNROLL];
#pragma unroll
                for (int u = 0; u < MD_UNROLL; ++u) pj[u] = __ldg(&pp[e[u] & MD_J_MASK]);
#pragma unroll
                for (int u = 0; u < MD_UNROLL; ++u) {
                    float dx, dy, dz;
                    disp<PER>(pi, pj[u], e[u] >> MD_J_BITS, sm_off, G, dx, dy, dz);
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * qu2;
                    if (k0 + u * TPA < n && r2 < a.rin2) {
                        // lane-interleaved rows: each lane owns rows lane, lane + TPA, ...
                        a.inner[(size_t)(m * TPA + lane) * S + s] = (int32_t)e[u];
                        if (r2 < Q.rc2) {
                            const float f = fa_val<IPOW>(Q, r2);
                            rho += f;
                            Ps = fmaf(f, f, Ps);
                        }
                        ++m;
                    }
                }
            }
            if (lane == 0) a.pin[s] = pi;
        } else {
            const int n = a.icnt[s];
            // the next batch's list entries are loaded while this batch is gathered and
            // summed (as in k_force), so only the gather's latency stays on the path
            const size_t rstep = (size_t)TPA * S;
            const int32_t *rowp = a.inner + (size_t)lane * S + s;
            unsigned en[MD_UNROLL];
#pragma unroll
            for (int u = 0; u < MD_UNROLL; ++u)
                en[u] = lane + u * TPA < n ? ld_stream(rowp + u * rstep) : (unsigned)s;
            rowp += MD_UNROLL * rstep;
            for (int k0 = lane; k0 < n; k0 += TPA * MD_UNROLL, rowp += MD_UNROLL * rstep) {
                unsigned e[MD_UNROLL];
#pragma unroll
                for (int u = 0; u < MD_UNROLL; ++u) {
                    e[u] = en[u];
                    en[u] = k0 + (u + MD_UNROLL) * TPA < n ? ld_stream(rowp + u * rstep) : (unsigned)s;
                }
                int4 pj[MD_UNROLL];
#pragma unroll
                for (int u = 0; u < MD_UNROLL; ++u) pj[u] = __ldg(&pp[e[u] & MD_J_MASK]);
#pragma unroll
                for (int u = 0; u < MD_UNROLL; ++u) {
                    float dx, dy, dz;
                    disp<PER>(pi, pj[u], e[u] >> MD_J_BITS, sm_off, G, dx, dy, dz);
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * qu2;
                    // padding entries (the atom itself) and entries now beyond rc drop out
                    const bool in = (e[u] & MD_J_MASK) != (unsigned)s && r2 < Q.rc2;
                    float f = fa_val<IPOW>(Q, in ? r2 : Q.rc2);
                    f = in ? f : 0.0f;
                    rho += f;
                    Ps = fmaf(f, f, Ps);
                }
            }
        }
    };
    if (per) work(BoolC<true>{}); else work(BoolC<false>{});
    int mmax = m;
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) {
        rho += __shfl_xor_sync(0xffffffffu, rho, o);
        Ps += __shfl_xor_sync(0xffffffffu, Ps, o);
        mmax = max(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
    }
    if (real && rebuild) {
        // rows of lanes with fewer entries are padded with the atom itself (skipped)
        for (int k = m; k < mmax; ++k) a.inner[(size_t)(k * TPA + lane) * S + s] = s;
        if (lane == 0) a.icnt[s] = mmax * TPA;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rebuild) a.st->inner_ok_next = 1;   // read by the next k_decide
        a.st->imax_fresh = rebuild;
    }
    double acc[2] = {0.0, 0.0};   // per-atom energies, summed over atoms in FP64
    if (real && lane == 0) {
        float F, Fp, M, Mp;
        Q.embed(rho, F, Fp);
        Q.mterm(Ps, M, Mp);
        a.fm32[s] = make_float2(Fp, 2.0f * Mp);   // (F', 2 M'): the force loop's factors
        acc[0] = F; acc[1] = M;
    }
    if (EN) cta_partials<2>(acc, a.part, a.max_blocks, blockIdx.x);
}

// Task 4b,c (Eq. (1) with the M term, Eqs. A6-A10; Morse Eqs. A5, A9) and Task 5 (the
// closing half kick, FP64).  The force on i from j is coef * (x_j - x_i), coef = [(F'_i +
// F'_j) f' + (M'_i + M'_j) 2 f f' + Phi'] / r, over the inner list; its entries beyond rc
// (~3 %) drop out by a select (a branch on the distance measured 10 % slower).  EN: the
// pair and Morse energies, the indenter load and the kinetic energy into the CTA partials
// (only the last step of an md_step call needs them).  integrate: 0 forces only; 1 a time
// step's Task 5, then the next step's Task 3 (drift) from the state just completed; 2 no
// kick (the forces of a state set from outside), then the next step's Task 3 from it.
template <int TPA, int IPOW, bool EN>
__global__ void __launch_bounds__(256, 5) k_force_mixed(DevArgs a, PotDev P, int integrate)
{
    __shared__ int4 sm_off[64];
    const int A = blockDim.x / TPA;
    const int g = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int s = blockIdx.x * A + g;
    const int r = a.tile_rep[(blockIdx.x * A) / MD_TILE];
    const RepDev &R = a.rep[r];
    fill_offsets(sm_off, R);
    __syncthreads();
    const Pot32 &Q = static_cast<const Pot32 &>(P.q);
    const bool real = (s - R.slot_off) < R.n_atoms;
    const size_t S = a.S;
    float gx = 0.f, gy = 0.f, gz = 0.f, ep = 0.f;
    float mx = 0.f, my = 0.f, mz = 0.f, em = 0.f;
    const int bn = buf_step(a), bo = bn ^ 1;   // the positions evaluated in bn; the drift goes to bo
    if (integrate && threadIdx.x == 0 && (A & 1) == 0) {
        // the epilogue's per-atom inputs of this CTA's atoms, on their way to L2 while the
        // pair loop runs (A even: every range starts and ends on a 16-byte boundary)
        const int s0 = blockIdx.x * A;
        const size_t S = a.S;
        for (int k = 0; k < 3; ++k) {
            prefetch_l2(a.xs[bn] + k * S + s0, A * 8u);
            prefetch_l2((integrate == 1 ? a.vh : a.v) + k * S + s0, A * 8u);
        }
        prefetch_l2(a.pb + s0, A * 16u);
        prefetch_l2(a.pin + s0, A * 16u);
    }
    const int4 *pp = a.p4[bn];
    const int4 pi = pp[s];
    const PairGeom G = pair_geom(R, pi.w);
    const float qu2 = a.qu * a.qu;   // r^2 from displacements in units of qu
    const bool per = __any_sync(0xffffffffu, real && G.xmask != 0u);
    if (TPA == 1) {   // this warp's inner-list rows (32 atoms: 128 B per row) on their way to L2
        const int nmax = __reduce_max_sync(0xffffffffu, real ? a.icnt[s] : 0);
        const int sw = s & ~31;
        for (int k = threadIdx.x & 31; k < nmax; k += 32) prefetch_l2(a.inner + (size_t)k * S + sw, 128u);
    }
    auto work = [&](auto PERC) {
        constexpr bool PER = decltype(PERC)::value;
        if (!real) return;
        const float2 fmi = a.fm32[s];
        const int n = a.icnt[s];
        // FU entries per lane per batch; the next batch's list entries are loaded while
        // this batch's neighbours are gathered and summed, so only the gather's latency
        // stays on each batch's path (2 entries: -2.5 % against 4 loaded together, which
        // with the look-ahead would spill under the register bound)
        constexpr int FU = 2;
        // row k of this lane at rowp + (k - lane) / TPA * rstep: advanced by increments
        const size_t rstep = (size_t)TPA * S;
        const int32_t *rowp = a.inner + (size_t)lane * S + s;
        unsigned en[FU];
#pragma unroll
        for (int u = 0; u < FU; ++u) en[u] = lane + u * TPA < n ? ld_stream(rowp + u * rstep) : (unsigned)s;
        rowp += FU * rstep;
        for (int k0 = lane; k0 < n; k0 += TPA * FU, rowp += FU * rstep) {
            unsigned e[FU];
#pragma unroll
            for (int u = 0; u < FU; ++u) {
                e[u] = en[u];
                en[u] = k0 + (u + FU) * TPA < n ? ld_stream(rowp + u * rstep) : (unsigned)s;
            }
            int4 pj[FU];
            float2 fmj[FU];
#pragma unroll
            for (int u = 0; u < FU; ++u) {
                const unsigned j = e[u] & MD_J_MASK;
                pj[u] = __ldg(&pp[j]);
                fmj[u] = __ldg(&a.fm32[j]);
            }
            // beta = 6: the batch's two pairs in packed FP32x2 arithmetic (a warp-uniform
            // path: an atom's last batch with one entry only computes its padding too)
            if (IPOW == 3 && FU == 2) {
                // a padding entry (the atom itself: r = 0, non-finite terms) is dropped by the
                // selects below, which never multiply it
                const bool real0 = (e[0] & MD_J_MASK) != (unsigned)s, real1 = (e[FU - 1] & MD_J_MASK) != (unsigned)s;
                float dx0, dy0, dz0, dx1, dy1, dz1;
                disp<PER>(pi, pj[0], e[0] >> MD_J_BITS, sm_off, G, dx0, dy0, dz0);
                disp<PER>(pi, pj[FU - 1], e[FU - 1] >> MD_J_BITS, sm_off, G, dx1, dy1, dz1);
                float2 R2, COEF, PH;
                pair_force6x2<EN>(Q, qu2, fmi, fmj[0], fmj[FU - 1], make_float2(dx0, dx1), make_float2(dy0, dy1),
                                  make_float2(dz0, dz1), R2, COEF, PH);
                const bool in0 = real0 && R2.x < Q.rc2, in1 = real1 && R2.y < Q.rc2;
                const float cw0 = in0 ? COEF.x : 0.0f, cw1 = in1 ? COEF.y : 0.0f;
                gx = fmaf(cw0, dx0, gx);
                gy = fmaf(cw0, dy0, gy);
                gz = fmaf(cw0, dz0, gz);
                gx = fmaf(cw1, dx1, gx);
                gy = fmaf(cw1, dy1, gy);
                gz = fmaf(cw1, dz1, gz);
                if (EN) {
                    ep += in0 ? PH.x : 0.0f;
                    ep += in1 ? PH.y : 0.0f;
                }
                continue;
            }
#pragma unroll
            for (int u = 0; u < FU; ++u) {
                float dx, dy, dz;
                disp<PER>(pi, pj[u], e[u] >> MD_J_BITS, sm_off, G, dx, dy, dz);
                if ((e[u] & MD_J_MASK) != (unsigned)s) {   // padding is the atom itself
                    // inner-list entries beyond rc (at most rc + inner skin) drop out by a
                    // select: their terms are finite
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * qu2;
                    const float rinv = rsqrt_nr(r2);
                    float f, df, ph, dph;
                    fa_phi<IPOW, EN>(Q, r2, rinv, f, df, ph, dph);
                    // [(F'_i + F'_j) + 2 (M'_i + M'_j) f] f' + Phi', over r
                    const float coef = fmaf(fmaf(fmi.y + fmj[u].y, f, fmi.x + fmj[u].x), df, dph) * rinv;
                    ph *= 0.5f;
                    const bool in = r2 < Q.rc2;
                    const float cw = in ? coef : 0.0f;
                    gx = fmaf(cw, dx, gx);
                    gy = fmaf(cw, dy, gy);
                    gz = fmaf(cw, dz, gz);
                    if (EN) ep += in ? ph : 0.0f;
                }
            }
        }
    };
    if (per) work(BoolC<true>{}); else work(BoolC<false>{});
    gx *= a.qu; gy *= a.qu; gz *= a.qu;   // the pair sums were taken over displacements in units of qu
    // Cr-C (Morse): summed by k_morse_mixed for the atoms with Cr-C neighbours
    if (real && lane == 0 && a.cntc[s] > 0) {
        const float4 fmo = a.fmorse[s];
        mx = fmo.x; my = fmo.y; mz = fmo.z; em = EN ? fmo.w : 0.0f;
    }
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
        mx += __shfl_xor_sync(0xffffffffu, mx, o);
        my += __shfl_xor_sync(0xffffffffu, my, o);
        mz += __shfl_xor_sync(0xffffffffu, mz, o);
        if (EN) {
            ep += __shfl_xor_sync(0xffffffffu, ep, o);
            em += __shfl_xor_sync(0xffffffffu, em, o);
        }
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // per-atom energies and load, summed over atoms in FP64
    unsigned long long d2bits = 0ull;
    unsigned ibits = 0u;
    if (real && lane == 0) {
        const double Fx = gx + mx, Fy = gy + my, Fz = gz + mz;
        a.F[s] = Fx; a.F[S + s] = Fy; a.F[2 * S + s] = Fz;
        double vx, vy, vz;
        if (integrate) {
            if (integrate == 1) {   // Task 5: v(t+dt) = v(t+dt/2) + a(t+dt) dt/2 (FP64)
                vx = a.vh[s]; vy = a.vh[S + s]; vz = a.vh[2 * S + s];
                if (!a.fixed[s]) {
                    const double hk = R.hk;
                    vx = fma(hk, Fx, vx); vy = fma(hk, Fy, vy); vz = fma(hk, Fz, vz);
                    a.v[s] = vx; a.v[S + s] = vy; a.v[2 * S + s] = vz;
                }
            } else {
                vx = a.v[s]; vy = a.v[S + s]; vz = a.v[2 * S + s];
            }
            // Task 3 of the next step, from the state just completed (x(t + 2 dt) in a
            // time step, x(t + dt) from a set state) to buffer bo, its rebuild test for the
            // k_decide that examines those positions, its inner-list test for the k_density
            // that evaluates them.  The next k_decide keeps it unless it rebuilds the lists.
            const double *x = a.xs[bn];
            drift_atom(a, R, s, pi.w, integrate == 1 ? a.rs[r].dthr2 : a.rs[r].dthr, x[s], x[S + s],
                       x[2 * S + s], vx, vy, vz, Fx, Fy, Fz, a.xs[bo], a.p4[bo], d2bits, ibits);
        } else {
            vx = a.v[s]; vy = a.v[S + s]; vz = a.v[2 * S + s];
        }
        if (EN) {
            acc[0] = ep; acc[1] = em; acc[2] = -mz;
            acc[3] = (0.5 / MD_ACC) * R.mass * (vx * vx + vy * vy + vz * vz);   // kinetic energy, FP64
        }
    }
    if (integrate) cta_max_disp(d2bits, ibits, &a.rs[r].d2b[bo], &a.st->imax_next);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->drift_ok = integrate != 0;
        if (integrate == 1) a.st->since_build += 1;
    }
    if (EN) cta_partials<4>(acc, a.part + 2 * (size_t)a.max_blocks, a.max_blocks, blockIdx.x);
}

// Task 4c for the mixed path (Eqs. A5, A9): one warp per atom with Cr-C neighbours (the
// queue built with the list), lanes over its entries; FP64 geometry of each pair, FP32
// potential; the atom's Morse force and energy go to fmorse[s], which k_force_mixed adds.
// The sums depend on the atom only, not on its place in the queue.
__global__ void __launch_bounds__(256) k_morse_mixed(DevArgs a, PotDev P)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int n_near = a.st->n_near;
    const Pot32 &Q = static_cast<const Pot32 &>(P.q);
    const size_t S = a.S, C = a.C;
    for (int qi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; qi < n_near; qi += nw) {
        const int s = a.near[qi];
        const int r = a.tile_rep[s / MD_TILE];
        const RepDev &R = a.rep[r];
        const int nc = a.cntc[s];
        const double *x = a.xs[buf_step(a)];   // x(t + dt), with the indenter at z_ind(t + dt)
        const double xi = x[s], yi = x[S + s], zi = x[2 * S + s];
        const double z_ind = a.rs[r].z_ind;
        float mx = 0.f, my = 0.f, mz = 0.f, em = 0.f;
        for (int k = lane; k < nc; k += 32) {
            const int c = __ldg(&a.nbrc[(size_t)k * S + s]);
            const double ddx = mi64(a.xc0[c] - xi, R.per[0], R.L[0]);
            const double ddy = mi64(a.xc0[C + c] - yi, R.per[1], R.L[1]);
            const double ddz = mi64(a.xc0[2 * C + c] + z_ind - zi, R.per[2], R.L[2]);
            const double y2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (y2 < P.rcm2) {
                const float yinv = rsqrtf((float)y2);
                float v, dv;
                Q.morse((float)y2 * yinv, v, dv);
                const float c1 = dv * yinv;
                mx = fmaf(c1, (float)ddx, mx);
                my = fmaf(c1, (float)ddy, my);
                mz = fmaf(c1, (float)ddz, mz);
                em += v;
            }
        }
        mx = warp_sum(mx); my = warp_sum(my); mz = warp_sum(mz); em = warp_sum(em);
        if (lane == 0) a.fmorse[s] = make_float4(mx, my, mz, em);
    }
}

// ============================================================================ Task 4, FP64

template <int TPA>
__global__ void __launch_bounds__(256) k_density_fp64(DevArgs a, PotDev P)
{
    const int A = blockDim.x / TPA;
    const int g = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int s = blockIdx.x * A + g;
    const RepDev &R = a.rep[a.tile_rep[(blockIdx.x * A) / MD_TILE]];
    const bool real = (s - R.slot_off) < R.n_atoms;
    const size_t S = a.S;
    double rho = 0.0, Ps = 0.0;
    const double *x = a.xs[buf_step(a)];
    if (real) {
        const double xi = x[s], yi = x[S + s], zi = x[2 * S + s];
        const int n = a.cnt[s];
        for (int k = lane; k < n; k += TPA) {
            const int j = (int)((unsigned)__ldg(&a.nbr[(size_t)k * S + s]) & MD_J_MASK);
            const double dx = mi64(x[j] - xi, R.per[0], R.L[0]);
            const double dy = mi64(x[S + j] - yi, R.per[1], R.L[1]);
            const double dz = mi64(x[2 * S + j] - zi, R.per[2], R.L[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.rc2) {
                double f, df;
                f_64(P, sqrt(r2), f, df);
                rho += f;
                Ps += f * f;
            }
        }
    }
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) {
        rho += __shfl_xor_sync(0xffffffffu, rho, o);
        Ps += __shfl_xor_sync(0xffffffffu, Ps, o);
    }
    double acc[2] = {0.0, 0.0};
    if (real && lane == 0) {
        double F, Fp, M, Mp;
        embed_64(P, rho, F, Fp);
        mterm_64(P, Ps, M, Mp);
        a.fm64[s] = make_double2(Fp, Mp);
        acc[0] = F; acc[1] = M;
    }
    cta_partials<2>(acc, a.part, a.max_blocks, blockIdx.x);
}

template <int TPA>
__global__ void __launch_bounds__(256) k_force_fp64(DevArgs a, PotDev P, int integrate)
{
    const int A = blockDim.x / TPA;
    const int g = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int s = blockIdx.x * A + g;
    const int r = a.tile_rep[(blockIdx.x * A) / MD_TILE];
    const RepDev &R = a.rep[r];
    const bool real = (s - R.slot_off) < R.n_atoms;
    const size_t S = a.S, C = a.C;
    double gx = 0.0, gy = 0.0, gz = 0.0, ep = 0.0;
    double mx = 0.0, my = 0.0, mz = 0.0, em = 0.0;
    const double *x = a.xs[buf_step(a)];
    if (real) {
        const double xi = x[s], yi = x[S + s], zi = x[2 * S + s];
        const double2 fmi = a.fm64[s];
        const int n = a.cnt[s];
        for (int k = lane; k < n; k += TPA) {
            const int j = (int)((unsigned)__ldg(&a.nbr[(size_t)k * S + s]) & MD_J_MASK);
            const double dx = mi64(x[j] - xi, R.per[0], R.L[0]);
            const double dy = mi64(x[S + j] - yi, R.per[1], R.L[1]);
            const double dz = mi64(x[2 * S + j] - zi, R.per[2], R.L[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.rc2) {
                const double2 fmj = a.fm64[j];
                const double rr = sqrt(r2);
                double f, df, ph, dph;
                f_64(P, rr, f, df);
                phi_64(P, rr, ph, dph);
                const double coef = ((fmi.x + fmj.x) * df + (fmi.y + fmj.y) * 2.0 * f * df + dph) / rr;
                gx += coef * dx; gy += coef * dy; gz += coef * dz;
                ep += 0.5 * ph;
            }
        }
        const int nc = a.cntc[s];
        if (nc > 0) {
            const double z_ind = a.rs[r].z_ind;
            for (int k = lane; k < nc; k += TPA) {
                const int c = __ldg(&a.nbrc[(size_t)k * S + s]);
                const double ddx = mi64(a.xc0[c] - xi, R.per[0], R.L[0]);
                const double ddy = mi64(a.xc0[C + c] - yi, R.per[1], R.L[1]);
                const double ddz = mi64(a.xc0[2 * C + c] + z_ind - zi, R.per[2], R.L[2]);
                const double y2 = ddx * ddx + ddy * ddy + ddz * ddz;
                if (y2 < P.rcm2) {
                    const double y = sqrt(y2);
                    double v, dv;
                    morse_64(P, y, v, dv);
                    mx += dv * ddx / y; my += dv * ddy / y; mz += dv * ddz / y;
                    em += v;
                }
            }
        }
    }
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
        ep += __shfl_xor_sync(0xffffffffu, ep, o);
        mx += __shfl_xor_sync(0xffffffffu, mx, o);
        my += __shfl_xor_sync(0xffffffffu, my, o);
        mz += __shfl_xor_sync(0xffffffffu, mz, o);
        em += __shfl_xor_sync(0xffffffffu, em, o);
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (real && lane == 0) {
        const double Fx = gx + mx, Fy = gy + my, Fz = gz + mz;
        a.F[s] = Fx; a.F[S + s] = Fy; a.F[2 * S + s] = Fz;
        const double *vs = integrate ? a.vh : a.v;   // v(t + dt/2) from k_verlet1, or the state
        double vx = vs[s], vy = vs[S + s], vz = vs[2 * S + s];
        if (integrate && !a.fixed[s]) {   // Task 5: v(t+dt) = v(t+dt/2) + a(t+dt) dt/2
            const double hk = 0.5 * R.dt * R.acc_per_f;
            vx += hk * Fx; vy += hk * Fy; vz += hk * Fz;
            a.v[s] = vx; a.v[S + s] = vy; a.v[2 * S + s] = vz;
        }
        acc[0] = ep; acc[1] = em; acc[2] = -mz;
        acc[3] = 0.5 * R.mass * (vx * vx + vy * vy + vz * vz) / MD_ACC;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.st->drift_ok = 0;   // no drift ahead on the FP64 path: k_verlet1 runs every step
        if (integrate) a.st->since_build += 1;
    }
    cta_partials<4>(acc, a.part + 2 * (size_t)a.max_blocks, a.max_blocks, blockIdx.x);
}

// ============================================================================ per-atom virial

// c d (x) d / 2 into w (xx yy zz xy xz yz): the pair term whose energy derivative is c r
template <class T>
__device__ __forceinline__ void add_vir(T (&w)[6], T c, T dx, T dy, T dz)
{
    const T h = c * (T)0.5;
    w[0] += h * dx * dx; w[1] += h * dy * dy; w[2] += h * dz * dz;
    w[3] += h * dx * dy; w[4] += h * dx * dz; w[5] += h * dy * dz;
}

// Per-atom virial (the potential part of per-atom stress times volume; Sec. 2.1 lists
// stresses among Task 4's outputs): every pair term of the energy depends on one distance r,
// the force on i from j is c (x_j - x_i) with c = (dE/dr) / r -- the coef of k_force_mixed --
// and each atom of the pair takes half of c (x_j - x_i) (x) (x_j - x_i); a Cr-C pair gives
// its half to the Cr atom.  Mixed precision: the inner list and pos4 of the state, FP32 pair
// terms as in k_force_mixed, the Cr-C pairs with FP64 geometry as in k_morse_mixed.
template <int TPA, int IPOW>
__global__ void __launch_bounds__(256) k_virial_mixed(DevArgs a, PotDev P)
{
    __shared__ int4 sm_off[64];
    const int A = blockDim.x / TPA;
    const int g = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int s = blockIdx.x * A + g;
    const int r = a.tile_rep[(blockIdx.x * A) / MD_TILE];
    const RepDev &R = a.rep[r];
    fill_offsets(sm_off, R);
    __syncthreads();
    const Pot32 &Q = static_cast<const Pot32 &>(P.q);
    const bool real = (s - R.slot_off) < R.n_atoms;
    const size_t S = a.S;
    const int b = buf_step(a);
    const int4 *pp = a.p4[b];
    const int4 pi = pp[s];
    const PairGeom G = pair_geom(R, pi.w);
    const bool per = __any_sync(0xffffffffu, real && G.xmask != 0u);
    float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto work = [&](auto PERC) {
        constexpr bool PER = decltype(PERC)::value;
        if (!real) return;
        const float2 fmi = a.fm32[s];
        const int n = a.icnt[s];
        for (int k = lane; k < n; k += TPA) {
            const unsigned e = (unsigned)__ldg(&a.inner[(size_t)k * S + s]);
            const unsigned j = e & MD_J_MASK;
            if (j == (unsigned)s) continue;   // padding
            float dx, dy, dz;
            disp<PER>(pi, __ldg(&pp[j]), e >> MD_J_BITS, sm_off, G, dx, dy, dz);
            dx *= a.qu; dy *= a.qu; dz *= a.qu;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(r2 < Q.rc2)) continue;
            const float2 fmj = __ldg(&a.fm32[j]);
            const float rinv = rsqrt_nr(r2);
            float f, df, ph, dph;
            fa_phi<IPOW, false>(Q, r2, rinv, f, df, ph, dph);
            const float coef = fmaf(fmaf(fmi.y + fmj.y, f, fmi.x + fmj.x), df, dph) * rinv;
            add_vir(w, coef, dx, dy, dz);
        }
    };
    if (per) work(BoolC<true>{}); else work(BoolC<false>{});
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
    if (!real || lane != 0) return;
    double W[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) W[k] = w[k];
    const int nc = a.cntc[s];
    if (nc > 0) {
        const double *x = a.xs[b];
        const double xi = x[s], yi = x[S + s], zi = x[2 * S + s];
        const double z_ind = a.rs[r].z_ind;
        const size_t C = a.C;
        for (int k = 0; k < nc; ++k) {
            const int c = __ldg(&a.nbrc[(size_t)k * S + s]);
            const double ddx = mi64(a.xc0[c] - xi, R.per[0], R.L[0]);
            const double ddy = mi64(a.xc0[C + c] - yi, R.per[1], R.L[1]);
            const double ddz = mi64(a.xc0[2 * C + c] + z_ind - zi, R.per[2], R.L[2]);
            const double y2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (y2 < P.rcm2) {
                const float yinv = rsqrtf((float)y2);
                float v, dv;
                Q.morse((float)y2 * yinv, v, dv);
                add_vir(W, (double)(dv * yinv), ddx, ddy, ddz);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) a.vir[k * S + s] = W[k];
}

// the same in FP64 over the Verlet list (pairs within rc), FP64 potential forms
template <int TPA>
__global__ void __launch_bounds__(256) k_virial_fp64(DevArgs a, PotDev P)
{
    const int A = blockDim.x / TPA;
    const int g = threadIdx.x / TPA, lane = threadIdx.x % TPA;
    const int s = blockIdx.x * A + g;
    const int r = a.tile_rep[(blockIdx.x * A) / MD_TILE];
    const RepDev &R = a.rep[r];
    const bool real = (s - R.slot_off) < R.n_atoms;
    const size_t S = a.S, C = a.C;
    const double *x = a.xs[buf_step(a)];
    double w[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (real) {
        const double xi = x[s], yi = x[S + s], zi = x[2 * S + s];
        const double2 fmi = a.fm64[s];
        const int n = a.cnt[s];
        for (int k = lane; k < n; k += TPA) {
            const int j = (int)((unsigned)__ldg(&a.nbr[(size_t)k * S + s]) & MD_J_MASK);
            const double dx = mi64(x[j] - xi, R.per[0], R.L[0]);
            const double dy = mi64(x[S + j] - yi, R.per[1], R.L[1]);
            const double dz = mi64(x[2 * S + j] - zi, R.per[2], R.L[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.rc2) {
                const double2 fmj = a.fm64[j];
                const double rr = sqrt(r2);
                double f, df, ph, dph;
                f_64(P, rr, f, df);
                phi_64(P, rr, ph, dph);
                add_vir(w, ((fmi.x + fmj.x) * df + (fmi.y + fmj.y) * 2.0 * f * df + dph) / rr, dx, dy, dz);
            }
        }
        const int nc = a.cntc[s];
        const double z_ind = a.rs[r].z_ind;
        for (int k = lane; k < nc; k += TPA) {
            const int c = __ldg(&a.nbrc[(size_t)k * S + s]);
            const double ddx = mi64(a.xc0[c] - xi, R.per[0], R.L[0]);
            const double ddy = mi64(a.xc0[C + c] - yi, R.per[1], R.L[1]);
            const double ddz = mi64(a.xc0[2 * C + c] + z_ind - zi, R.per[2], R.L[2]);
            const double y2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (y2 < P.rcm2) {
                const double y = sqrt(y2);
                double v, dv;
                morse_64(P, y, v, dv);
                add_vir(w, dv / y, ddx, ddy, ddz);
            }
        }
    }
#pragma unroll
    for (int o = TPA / 2; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] += __shfl_xor_sync(0xffffffffu, w[k], o);
    if (real && lane == 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) a.vir[k * S + s] = w[k];
}

// per-replica sums of the CTA partials in a fixed order.  gridDim.x (<= MD_RED_CHUNKS, fixed
// for a handle) CTAs per replica each sum a contiguous run of the partials (thread t adds blocks t, t + B, ... of all six
// terms together; the lanes of a warp by a fixed shuffle tree; thread 0 the warp sums in
// warp order) into rsum; the CTA that finishes last (a counter per replica, after a fence)
// adds the chunk sums in chunk order and resets the counter.  Which CTA finishes last does
// not change a bit of the result.
__global__ void __launch_bounds__(64) k_reduce(DevArgs a, int atoms_per_block)
{
    const int r = blockIdx.y, ch = blockIdx.x, nch = gridDim.x;
    const RepDev &R = a.rep[r];
    const int b0 = R.slot_off / atoms_per_block, b1 = (R.slot_off + R.n_slots) / atoms_per_block;
    const int per = (b1 - b0 + nch - 1) / nch;
    const int c0 = min(b1, b0 + ch * per), c1 = min(b1, c0 + per);
    const size_t stride = (size_t)a.max_blocks;
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = c0 + threadIdx.x; b < c1; b += blockDim.x) {
#pragma unroll
        for (int t = 0; t < 6; ++t) acc[t] += a.part[t * stride + b];
    }
#pragma unroll
    for (int t = 0; t < 6; ++t)
        for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_down_sync(0xffffffffu, acc[t], o);
    __shared__ double sm[32][6];
    __shared__ int last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < 6; ++t) sm[wid][t] = acc[t];
    }
    __syncthreads();
    double *mine = a.rsum + ((size_t)r * nch + ch) * 6;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < 6; ++t) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sm[w][t];
            mine[t] = s;
        }
        __threadfence();   // the chunk sums are visible before the count says so
        last = atomicAdd(&a.rs[r].rctr, 1) == nch - 1;
    }
    __syncthreads();
    if (!last) return;   // CTA-uniform
    __threadfence();
    // the chunk sums (read past L1, where another CTA's writes are not) into shared memory
    // by many threads at once, then added in chunk order
    __shared__ double cs[MD_RED_CHUNKS * 6];
    const double *all = a.rsum + (size_t)r * nch * 6;
    for (int i = threadIdx.x; i < nch * 6; i += blockDim.x) cs[i] = __ldcg(&all[i]);
    __syncthreads();
    __shared__ double out[6];
    if (threadIdx.x < 6) {   // one thread per term (FP64 adds are slow on this part: in parallel)
        const int t = threadIdx.x;
        double s = 0.0;
        for (int k = 0; k < nch; ++k) s += cs[k * 6 + t];
        out[t] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        RepEnergy &E = a.en[r];
        E.embed = out[0]; E.mterm = out[1]; E.pair = out[2]; E.morse = out[3];
        E.load = out[4]; E.kinetic = out[5];
        a.rs[r].rctr = 0;
    }
}

inline unsigned nblk(long n, int b) { return (unsigned)((n + b - 1) / b); }

static int device_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        n = 0;
    return std::max(1, n);
}

// grids of the one-warp-per-atom Cr-C kernels (their atom count is known only on the
// device).  k_nbrc_near: every CTA the SMs hold at once; k_morse_mixed: 2 CTAs per SM, as
// it runs beside k_density in the step graphs (a full grid there cost the batch of 256
// replicas 2 % of its step)
template <class K>
static unsigned full_grid(K kernel, int block)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0) != cudaSuccess || occ < 1) occ = 1;
    return (unsigned)(occ * device_sms());
}

static unsigned morse_grid() { return (unsigned)(2 * device_sms()); }

}  // namespace

// ============================================================================ launchers

cudaError_t launch_decide(const DevArgs &a, int mode, int use_cond, cudaGraphConditionalHandle h, cudaStream_t s,
                          cudaGraphConditionalHandle hv)
{
    k_decide<<<1, 256, 0, s>>>(a, mode, use_cond, h, hv);
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const DevArgs &a, cudaStream_t s)
{
    const int B = 256;
    k_zero_i32<<<nblk(a.total_cells, B), B, 0, s>>>(a.cell_count, a.total_cells);
    k_zero_i32<<<nblk(a.total_cells, B), B, 0, s>>>(a.cell_fill, a.total_cells);
    k_bin<<<nblk(a.S, B), B, 0, s>>>(a);
    const int SB = 512, per_block = 2 * SB;
    int nb = (int)nblk(a.total_cells, per_block);
    k_scan1<<<nb, SB, SB * sizeof(int32_t), s>>>(a.cell_count, a.cell_start, a.scan_blk, a.total_cells);
    k_scan2<<<1, 1024, 1024 * sizeof(int32_t), s>>>(a.scan_blk, nb);
    k_scan3<<<nblk(a.total_cells, B), B, 0, s>>>(a, per_block);
    k_scatter<<<nblk(a.S, B), B, 0, s>>>(a);
    k_cellsort<<<nblk(a.total_cells, B), B, 0, s>>>(a);
    k_gather<<<nblk(a.S, B), B, 0, s>>>(a);
    k_copyback<<<nblk(a.S, B), B, 0, s>>>(a);
    k_nbr<<<nblk(a.S, 128), 128, 0, s>>>(a);
    k_nbrc<<<nblk(a.S, 128), 128, 0, s>>>(a);
    k_nbrc_near<<<full_grid(k_nbrc_near, 256), 256, 0, s>>>(a);
    k_build_done<<<1, 256, 0, s>>>(a);
    if (a.debug) {
        k_zero_chk<<<1, 32, 0, s>>>(a);
        k_check_lists<<<nblk(a.S, 128), 128, 0, s>>>(a, a.cut);
    }
    return cudaGetLastError();
}

cudaError_t launch_check_lists(const DevArgs &a, double radius, cudaStream_t s)
{
    k_zero_chk<<<1, 32, 0, s>>>(a);
    k_check_lists<<<nblk(a.S, 128), 128, 0, s>>>(a, radius > 0.0 ? radius : a.cut);
    return cudaGetLastError();
}

cudaError_t launch_verlet1(const DevArgs &a, cudaStream_t s)
{
    k_verlet1<<<a.S / MD_TILE, MD_TILE, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_drift_prep(const DevArgs &a, cudaStream_t s)
{
    k_drift_prep<<<1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_state_set(const DevArgs &a, int r, int slot_off, int n, double z_ind, long long step,
                             const double *stage, cudaStream_t s)
{
    k_state_prep<<<1, 32, 0, s>>>(a, r, z_ind, step);
    if (n > 0) k_state_scan<<<nblk(n, 256), 256, 0, s>>>(a, r, slot_off, n, stage);
    k_state_need<<<1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <int TPA>
static void dens_t(const DevArgs &a, const PotDev &p, int block, int en, cudaStream_t s)
{
    int A = block / TPA;
    if (a.mixed) {
        if (p.q.ipow == 3) {   // beta = 6
            if (en) k_density_mixed<TPA, 3, true><<<a.S / A, block, 0, s>>>(a, p);
            else k_density_mixed<TPA, 3, false><<<a.S / A, block, 0, s>>>(a, p);
        } else {
            if (en) k_density_mixed<TPA, 0, true><<<a.S / A, block, 0, s>>>(a, p);
            else k_density_mixed<TPA, 0, false><<<a.S / A, block, 0, s>>>(a, p);
        }
    }
    else {
        k_density_fp64<TPA><<<a.S / A, block, 0, s>>>(a, p);
    }
}

template <int TPA>
static void force_t(const DevArgs &a, const PotDev &p, int block, int integ, int en, cudaStream_t s)
{
    int A = block / TPA;
    if (a.mixed) {
        if (p.q.ipow == 3) {
            if (en) k_force_mixed<TPA, 3, true><<<a.S / A, block, 0, s>>>(a, p, integ);
            else k_force_mixed<TPA, 3, false><<<a.S / A, block, 0, s>>>(a, p, integ);
        } else {
            if (en) k_force_mixed<TPA, 0, true><<<a.S / A, block, 0, s>>>(a, p, integ);
            else k_force_mixed<TPA, 0, false><<<a.S / A, block, 0, s>>>(a, p, integ);
        }
    }
    else {
        k_force_fp64<TPA><<<a.S / A, block, 0, s>>>(a, p, integ);
    }
}

cudaError_t launch_density(const DevArgs &a, const PotDev &p, const LaunchCfg &c, int energies, cudaStream_t s)
{
    switch (c.tpa) {
    case 1: dens_t<1>(a, p, c.block, energies, s); break;
    case 2: dens_t<2>(a, p, c.block, energies, s); break;
    case 4: dens_t<4>(a, p, c.block, energies, s); break;
    default: dens_t<8>(a, p, c.block, energies, s); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_morse(const DevArgs &a, const PotDev &p, cudaStream_t s)
{
    if (a.mixed) k_morse_mixed<<<morse_grid(), 256, 0, s>>>(a, p);
    return cudaGetLastError();
}

cudaError_t launch_force(const DevArgs &a, const PotDev &p, const LaunchCfg &c, int integrate, int energies,
                         cudaStream_t s)
{
    return launch_force_split(a, p, c, integrate, energies, 1, s);
}

cudaError_t launch_force_split(const DevArgs &a, const PotDev &p, const LaunchCfg &c, int integrate, int energies,
                               int with_morse, cudaStream_t s)
{
    if (with_morse && a.mixed) k_morse_mixed<<<morse_grid(), 256, 0, s>>>(a, p);
    switch (c.tpa) {
    case 1: force_t<1>(a, p, c.block, integrate, energies, s); break;
    case 2: force_t<2>(a, p, c.block, integrate, energies, s); break;
    case 4: force_t<4>(a, p, c.block, integrate, energies, s); break;
    default: force_t<8>(a, p, c.block, integrate, energies, s); break;
    }
    return cudaGetLastError();
}

template <int TPA>
static void vir_t(const DevArgs &a, const PotDev &p, int block, cudaStream_t s)
{
    const int A = block / TPA;
    if (a.mixed) {
        if (p.q.ipow == 3) k_virial_mixed<TPA, 3><<<a.S / A, block, 0, s>>>(a, p);
        else k_virial_mixed<TPA, 0><<<a.S / A, block, 0, s>>>(a, p);
    } else {
        k_virial_fp64<TPA><<<a.S / A, block, 0, s>>>(a, p);
    }
}

cudaError_t launch_virial(const DevArgs &a, const PotDev &p, const LaunchCfg &c, cudaStream_t s)
{
    switch (c.tpa) {
    case 1: vir_t<1>(a, p, c.block, s); break;
    case 2: vir_t<2>(a, p, c.block, s); break;
    case 4: vir_t<4>(a, p, c.block, s); break;
    default: vir_t<8>(a, p, c.block, s); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const DevArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    // chunks per replica: one per ~32 CTA partials of the largest replica (1 .. MD_RED_CHUNKS):
    // 256 small replicas would otherwise launch 32 768 CTAs with a partial or none each
    const int apb = c.block / c.tpa;
    const int parts = (c.max_rep_slots + apb - 1) / apb + 1;
    const int nch = std::min(MD_RED_CHUNKS, std::max(1, (parts + 31) / 32));
    k_reduce<<<dim3(nch, a.n_rep), 64, 0, s>>>(a, apb);
    return cudaGetLastError();
}

// ============================================================================ md_forces_small

// The analytic fields of md_build_pot (fill_forms), without tables.
int md_pot_forms(const md_params *p, PotDev *P, char *err, size_t errlen)
{
    memset(P, 0, sizeof(*P));
    if (!(p->r_e > 0 && p->f_e > 0 && p->rho_e > 0 && p->P_e > 0 && p->y_eq > 0 && p->rc > 0 && p->rc_morse > 0)) {
        snprintf(err, errlen, "md_params: r_e, f_e, rho_e, P_e, y_eq, rc, rc_morse must be > 0");
        return MD_ERR_ARG;
    }
    if (p->tabulated) {
        snprintf(err, errlen, "md_forces_small evaluates the analytic forms: params->tabulated must be 0");
        return MD_ERR_ARG;
    }
    HostPot H;
    fill_forms(p, P, H);
    P->tabulated = 0;
    return MD_OK;
}

namespace {

constexpr size_t SMALL_SCRATCH_DOUBLES = 2 * (size_t)MD_SMALL_MAX_ATOMS + 4 * (size_t)MD_SMALL_MAX_BLOCKS;
static_assert(SMALL_SCRATCH_DOUBLES * 8 == MD_SMALL_SCRATCH_BYTES, "scratch size in md.h");

// the scratch of md_forces_small (one per device; see md.h for sharing rules)
static __device__ __align__(256) double g_small_scratch[SMALL_SCRATCH_DOUBLES];

__device__ __forceinline__ double mi_any(double d, int per, double L, double iL)
{
    return per ? d - L * rint(d * iL) : d;
}

// rho_i, P_i over all j != i within rc (Eqs. A2, A3); F'(rho_i), M'(P_i) to scratch,
// F(rho_i), M(P_i) into the CTA's sums
__global__ void __launch_bounds__(MD_SMALL_BLOCK) k_small_density(SmallArgs g, PotDev P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    if (i < g.n) {
        const double xi = g.x[3 * i], yi = g.x[3 * i + 1], zi = g.x[3 * i + 2];
        double rho = 0.0, Ps = 0.0;
        for (int j = 0; j < g.n; ++j) {
            if (j == i) continue;
            const double dx = mi_any(g.x[3 * j] - xi, g.per[0], g.L[0], g.iL[0]);
            const double dy = mi_any(g.x[3 * j + 1] - yi, g.per[1], g.L[1], g.iL[1]);
            const double dz = mi_any(g.x[3 * j + 2] - zi, g.per[2], g.L[2], g.iL[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.rc2) {
                double f, df;
                f_64(P, sqrt(r2), f, df);
                rho += f;
                Ps += f * f;
            }
        }
        double F, Fp, M, Mp;
        embed_64(P, rho, F, Fp);
        mterm_64(P, Ps, M, Mp);
        g.fm[2 * i] = Fp;
        g.fm[2 * i + 1] = Mp;
        acc[0] = F; acc[1] = M;
    }
    cta_partials<2>(acc, g.part, g.nb, blockIdx.x);
}

// forces (Eq. (1) with the M term, Morse Eq. A5) and the pair / Morse energies
__global__ void __launch_bounds__(MD_SMALL_BLOCK) k_small_force(SmallArgs g, PotDev P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double acc[2] = {0.0, 0.0};
    if (i < g.n) {
        const double xi = g.x[3 * i], yi = g.x[3 * i + 1], zi = g.x[3 * i + 2];
        const double fpi = g.fm[2 * i], mpi = g.fm[2 * i + 1];
        double gx = 0.0, gy = 0.0, gz = 0.0, ep = 0.0, em = 0.0;
        for (int j = 0; j < g.n; ++j) {
            if (j == i) continue;
            const double dx = mi_any(g.x[3 * j] - xi, g.per[0], g.L[0], g.iL[0]);
            const double dy = mi_any(g.x[3 * j + 1] - yi, g.per[1], g.L[1], g.iL[1]);
            const double dz = mi_any(g.x[3 * j + 2] - zi, g.per[2], g.L[2], g.iL[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < P.rc2) {
                const double rr = sqrt(r2);
                double f, df, ph, dph;
                f_64(P, rr, f, df);
                phi_64(P, rr, ph, dph);
                const double coef = ((fpi + g.fm[2 * j]) * df + (mpi + g.fm[2 * j + 1]) * 2.0 * f * df + dph) / rr;
                gx += coef * dx; gy += coef * dy; gz += coef * dz;
                ep += 0.5 * ph;
            }
        }
        for (int c = 0; c < g.n_c; ++c) {
            const double dx = mi_any(g.xc[3 * c] - xi, g.per[0], g.L[0], g.iL[0]);
            const double dy = mi_any(g.xc[3 * c + 1] - yi, g.per[1], g.L[1], g.iL[1]);
            const double dz = mi_any(g.xc[3 * c + 2] - zi, g.per[2], g.L[2], g.iL[2]);
            const double y2 = dx * dx + dy * dy + dz * dz;
            if (y2 < P.rcm2) {
                const double y = sqrt(y2);
                double v, dv;
                morse_64(P, y, v, dv);
                gx += dv * dx / y; gy += dv * dy / y; gz += dv * dz / y;
                em += v;
            }
        }
        g.F[3 * i] = gx; g.F[3 * i + 1] = gy; g.F[3 * i + 2] = gz;
        acc[0] = ep; acc[1] = em;
    }
    cta_partials<2>(acc, g.part + 2 * (size_t)g.nb, g.nb, blockIdx.x);
}

// the four energies: CTA sums added in block order by one thread each
__global__ void k_small_energy(SmallArgs g)
{
    const int t = threadIdx.x;   // 0 embed, 1 mterm, 2 pair, 3 morse in part
    if (t >= 4) return;
    double s = 0.0;
    for (int b = 0; b < g.nb; ++b) s += g.part[(size_t)t * g.nb + b];
    const int slot[4] = {0, 2, 1, 3};   // -> embed, pair, mterm, morse
    g.energy[slot[t]] = s;
}

}  // namespace

cudaError_t small_setup(double **scratch, size_t *n_doubles)
{
    *n_doubles = SMALL_SCRATCH_DOUBLES;
    cudaError_t e = cudaGetSymbolAddress((void **)scratch, g_small_scratch);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_small_density)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, k_small_force)) != cudaSuccess) return e;
    return cudaFuncGetAttributes(&fa, k_small_energy);
}

cudaError_t launch_small(const SmallArgs &g, const PotDev &P, cudaStream_t s)
{
    k_small_density<<<g.nb, MD_SMALL_BLOCK, 0, s>>>(g, P);
    k_small_force<<<g.nb, MD_SMALL_BLOCK, 0, s>>>(g, P);
    k_small_energy<<<1, 32, 0, s>>>(g);
    return cudaGetLastError();
}
