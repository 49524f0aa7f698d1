// Stable neo-Hookean tetrahedra: energy, gradient and the analytically projected Hessian.
//
// The paper's deformables use the Stable neo-Hookean energy (Sec. 8) with the analytic
// eigensystems of isotropic distortion energies it cites (Sec. 2, "Eigen Analysis"):
//   Psi = mu/2 (I2 - 3) + lam/2 (J - alpha)^2 - mu/2 log(I2 + 1),
//   I2 = ||F||^2, J = det F, alpha = 1 + mu/lam - mu/(4 lam).
// Per element (one thread): F = Ds Dm^-1, a rotation-variant SVD F = U diag(s) V^T
// (cyclic Jacobi on F^T F, then Gram-Schmidt on F V; s2 may be negative for an inverted
// element), and the nine eigenpairs of d2Psi/dF2 in closed form:
//   twist (i,j; k the third index):  mu(1 - 1/(I2+1)) + lam (J - alpha) s_k,  U (e_i e_j^T - e_j e_i^T) V^T / sqrt2
//   flip  (i,j):                     mu(1 - 1/(I2+1)) - lam (J - alpha) s_k,  U (e_i e_j^T + e_j e_i^T) V^T / sqrt2
//   scaling: eigenpairs (l, a) of the 3x3 matrix d2Psi/ds_i ds_j,            U diag(a) V^T
// The projected block is scale * vol * sum over modes with l > 0 of l w w^T, w = dF/dx^T vec(Q),
// where dF/dx^T maps a 3x3 G to forces (G Dm^-T columns on vertices 1..3, minus their sum on 0).
// It is formed per pair of vertices in the singular basis (U M U^T, M from the clamped twist /
// flip eigenvalues and the projected scaling block, which is the block itself where it is
// positive definite); the float64 Jacobi starts from a float32 pre-rotation.
// Energy and gradient are computed in float64 for both precisions; the projected Hessian in the
// precision it is stored in (float64, or float32 for the mixed form, whose blocks are float32).
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "context.cuh"
#include "scan.cuh"

namespace gipc {
namespace {

struct ElasticConst {
    double mu, lam, alpha, scale;
};

// Arithmetic-type constants of the Hessian projection.
template <typename CT>
struct Num;
template <>
struct Num<double> {
    static constexpr double jacobi_tol = 1e-34;   // off-diagonal^2 / diagonal^2 that ends the sweeps
    static constexpr double tiny = 1e-300;
    static constexpr double rel = 1e-14;
};
template <>
struct Num<float> {
    static constexpr float jacobi_tol = 1e-14f;
    static constexpr float tiny = 1e-35f;
    static constexpr float rel = 1e-6f;
};

// One Jacobi rotation zeroing a[p][q] of a symmetric 3x3 matrix, accumulating into v.
template <int P, int Q, typename CT>
__device__ __forceinline__ void jacobi_rot(CT (&a)[3][3], CT (&v)[3][3]) {
    constexpr int R = 3 - P - Q;
    const CT apq = a[P][Q];
    if (apq == CT(0)) return;
    // The angle phi (|phi| <= pi/4) with tan(2 phi) = rho / tau, tau = a_qq - a_pp, rho = 2 a_pq:
    // cos(2 phi) = |tau| / h and sin(2 phi) = sign(tau) rho / h with h = sqrt(tau^2 + rho^2), and
    // with u = cos^2(phi) = (1 + cos(2 phi)) / 2 in [1/2, 1]: t = tan(phi) = sin(2 phi) / (2 u),
    // c = sqrt(u), s = t c.  Two reciprocal square roots and no division or square root (on
    // GB300 each float64 division or square root is a sequence of several FP64 instructions).
    // In float32 the same t comes from a division and a square root (cheap there, and exact for
    // subnormal arguments, which the reciprocal square root is not).
    const CT tau = a[Q][Q] - a[P][P], rho = CT(2) * apq;
    const CT hh = tau * tau + rho * rho;
    CT t, c;
    if constexpr (std::is_same<CT, double>::value) {
        if (!(hh > CT(0))) return;   // both below the square root of the smallest subnormal
        const CT ih = rsqrt(hh);
        const CT u = CT(0.5) + CT(0.5) * (fabs(tau) * ih);
        const CT iu = rsqrt(u);
        t = (CT(0.5) * ((tau >= CT(0) ? rho : -rho) * ih)) * (iu * iu);
        c = u * iu;
    } else {
        // (equal diagonal entries and an off-diagonal entry whose square underflows: nothing to
        // rotate at this precision, and the quotient would be 0 / 0)
        const CT den = fabs(tau) + sqrt(hh);
        if (!(den > CT(0))) return;
        t = (tau >= CT(0) ? rho : -rho) / den;
        c = rsqrt(t * t + CT(1));
    }
    const CT s = t * c;
    a[P][P] -= t * apq;
    a[Q][Q] += t * apq;
    a[P][Q] = a[Q][P] = CT(0);
    const CT arp = a[R][P], arq = a[R][Q];
    a[R][P] = a[P][R] = c * arp - s * arq;
    a[R][Q] = a[Q][R] = s * arp + c * arq;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const CT vp = v[r][P], vq = v[r][Q];
        v[r][P] = c * vp - s * vq;
        v[r][Q] = s * vp + c * vq;
    }
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi; eigenvalues on the
// diagonal of a, eigenvectors in the columns of v.
template <typename CT>
__device__ __forceinline__ void jacobi3(CT (&a)[3][3], CT (&v)[3][3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) v[r][c] = r == c ? CT(1) : CT(0);
    for (int sweep = 0; sweep < 12; ++sweep) {
        const CT off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const CT dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (!(off > Num<CT>::jacobi_tol * dia)) break;
        jacobi_rot<0, 1>(a, v);
        jacobi_rot<0, 2>(a, v);
        jacobi_rot<1, 2>(a, v);
    }
}

template <typename CT>
__device__ __forceinline__ void cross(const CT* a, const CT* b, CT* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Rotation-variant SVD: F = U diag(s) V^T with det U = det V = 1, s0 >= s1 >= |s2|.
template <typename CT>
__device__ void svd3(const CT (&F)[3][3], CT (&U)[3][3], CT (&s)[3], CT (&V)[3][3]) {
    CT S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
    CT W[3][3];
    if constexpr (std::is_same<CT, double>::value) {
        // float32 pre-rotation: Jacobi in float32 (on the FP32 pipe) gives eigenvectors to about
        // 1e-7; made orthonormal again in float64 they turn S into W0^T S W0 with off-diagonal
        // entries of about 1e-7 |S|, which the float64 sweeps (quadratically convergent) finish in
        // one or two sweeps instead of three or four.  Outside float32's range: no pre-rotation.
        CT W0[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
        const float tr = (float)((S[0][0] + S[1][1]) + S[2][2]);
        if (tr > 1e-30f && tr < 1e30f) {
            float Sf[3][3], Wf[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Sf[i][j] = (float)S[i][j];
            jacobi3(Sf, Wf);
            // Gram-Schmidt on the columns in float64, third column as the cross product
            CT a0[3] = {Wf[0][0], Wf[1][0], Wf[2][0]}, a1[3] = {Wf[0][1], Wf[1][1], Wf[2][1]}, a2[3];
            const CT i0 = rsqrt(a0[0] * a0[0] + a0[1] * a0[1] + a0[2] * a0[2]);
#pragma unroll
            for (int r = 0; r < 3; ++r) a0[r] *= i0;
            const CT p01 = a0[0] * a1[0] + a0[1] * a1[1] + a0[2] * a1[2];
#pragma unroll
            for (int r = 0; r < 3; ++r) a1[r] -= p01 * a0[r];
            const CT i1 = rsqrt(a1[0] * a1[0] + a1[1] * a1[1] + a1[2] * a1[2]);
#pragma unroll
            for (int r = 0; r < 3; ++r) a1[r] *= i1;
            cross(a0, a1, a2);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                W0[r][0] = a0[r];
                W0[r][1] = a1[r];
                W0[r][2] = a2[r];
            }
            // S <- W0^T S W0 (symmetric)
            CT T[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) T[i][j] = S[i][0] * W0[0][j] + S[i][1] * W0[1][j] + S[i][2] * W0[2][j];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j)
                    S[i][j] = S[j][i] = W0[0][i] * T[0][j] + W0[1][i] * T[1][j] + W0[2][i] * T[2][j];
        }
        CT W1[3][3];
        jacobi3(S, W1);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) W[i][j] = W0[i][0] * W1[0][j] + W0[i][1] * W1[1][j] + W0[i][2] * W1[2][j];
    } else {
        jacobi3(S, W);
    }
    CT ev[3] = {S[0][0], S[1][1], S[2][2]};
    int o[3] = {0, 1, 2};
    // sort descending
    if (ev[o[0]] < ev[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
    if (ev[o[1]] < ev[o[2]]) { int t = o[1]; o[1] = o[2]; o[2] = t; }
    if (ev[o[0]] < ev[o[1]]) { int t = o[0]; o[0] = o[1]; o[1] = t; }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) V[r][c] = o[c] == 0 ? W[r][0] : (o[c] == 1 ? W[r][1] : W[r][2]);
    CT v0[3] = {V[0][0], V[1][0], V[2][0]}, v1[3] = {V[0][1], V[1][1], V[2][1]}, v2[3];
    cross(v0, v1, v2);  // third column = v0 x v1 makes V a rotation
#pragma unroll
    for (int r = 0; r < 3; ++r) V[r][2] = v2[r];
    // B = F V
    CT B[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) B[i][j] = F[i][0] * V[0][j] + F[i][1] * V[1][j] + F[i][2] * V[2][j];
    // Column norm n and 1/n: in float64 as |b|^2 rsqrt(|b|^2) and rsqrt(|b|^2) (one FP64 sequence
    // instead of a square root and a division), in float32 by a square root and a division.
    auto norm_inv = [](CT nn, CT& nrm, CT& inv) {
        if constexpr (std::is_same<CT, double>::value) {
            inv = nn > CT(0) ? rsqrt(nn) : CT(0);
            nrm = nn * inv;
        } else {
            nrm = sqrt(nn);
            inv = nrm > CT(0) ? CT(1) / nrm : CT(0);
        }
    };
    CT u0[3] = {B[0][0], B[1][0], B[2][0]};
    CT n0, i0;
    norm_inv(u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2], n0, i0);
    if (n0 > CT(0)) {
#pragma unroll
        for (int r = 0; r < 3; ++r) u0[r] *= i0;
    } else {
        u0[0] = CT(1); u0[1] = CT(0); u0[2] = CT(0);
    }
    CT b1[3] = {B[0][1], B[1][1], B[2][1]};
    const CT p = u0[0] * b1[0] + u0[1] * b1[1] + u0[2] * b1[2];
    CT u1[3] = {b1[0] - p * u0[0], b1[1] - p * u0[1], b1[2] - p * u0[2]};
    CT n1, i1;
    norm_inv(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2], n1, i1);
    if (n1 > Num<CT>::tiny && n1 > Num<CT>::rel * n0) {
#pragma unroll
        for (int r = 0; r < 3; ++r) u1[r] *= i1;
    } else {  // any unit vector orthogonal to u0
        const CT ax = fabs(u0[0]), ay = fabs(u0[1]), az = fabs(u0[2]);
        CT e[3] = {CT(0), CT(0), CT(0)};
        if (ax <= ay && ax <= az) e[0] = CT(1);
        else if (ay <= az) e[1] = CT(1);
        else e[2] = CT(1);
        cross(u0, e, u1);
        const CT m = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
#pragma unroll
        for (int r = 0; r < 3; ++r) u1[r] /= m;
        n1 = u1[0] * b1[0] + u1[1] * b1[1] + u1[2] * b1[2];
    }
    CT u2[3];
    cross(u0, u1, u2);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        U[r][0] = u0[r];
        U[r][1] = u1[r];
        U[r][2] = u2[r];
    }
    s[0] = n0;
    s[1] = n1;
    s[2] = u2[0] * B[0][2] + u2[1] * B[1][2] + u2[2] * B[2][2];
}

// G (3x3) -> w (12): forces G Dm^-T on vertices 1..3, minus their sum on vertex 0.
template <typename CT>
__device__ __forceinline__ void map_to_x(const CT (&G)[3][3], const CT (&Dmi)[3][3], CT (&w)[12]) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        CT s = CT(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // (G Dm^-T)[r][a] = sum_c G[r][c] Dmi[a][c]
            const CT h = G[r][0] * Dmi[a][0] + G[r][1] * Dmi[a][1] + G[r][2] * Dmi[a][2];
            w[3 * (a + 1) + r] = h;
            s += h;
        }
        w[r] = -s;
    }
}

// The Hessian layout is a run-time flag (not a template parameter) so that both layouts run the
// same compiled arithmetic and hold bit-identical values.  With `live` (per scene, the scene of
// each vertex in vscene) the elements of scenes left out get zero outputs without evaluation.
template <int PREC>
__global__ void __launch_bounds__(128)
eval_tets_kernel(const double* __restrict__ x, int64_t n, const int32_t* __restrict__ tets, int64_t T,
                 const double* __restrict__ Dm_inv, const double* __restrict__ vol, const ElasticConst K,
                 double* __restrict__ energy, double* __restrict__ grad, void* __restrict__ hess_v, bool blocks,
                 const int32_t* __restrict__ vscene, const int32_t* __restrict__ live) {
    using HT = typename std::conditional<PREC == GIPC_FP64, double, float>::type;
    HT* __restrict__ hess = static_cast<HT*>(hess_v);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int32_t vid[4];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        vid[a] = __ldg(tets + a * T + t);
        if (vid[a] < 0 || vid[a] >= n) ok = false;
    }
    if (!ok) {
        if (energy) energy[t] = 0.0;
        return;
    }
    if (live && !live[vscene[vid[0]]]) {
        if (energy) energy[t] = 0.0;
        if (grad) {
#pragma unroll
            for (int j = 0; j < 12; ++j) grad[j * T + t] = 0.0;
        }
        if (hess) {
            HT* const z0 = blocks ? hess + t * 144 : hess + t;
            const int64_t zs = blocks ? 1 : T;
            for (int j = 0; j < 144; ++j) z0[j * zs] = HT(0);
        }
        return;
    }
    double X[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int r = 0; r < 3; ++r) X[a][r] = __ldg(x + r * n + vid[a]);
    double Dmi[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Dmi[i][j] = __ldg(Dm_inv + (3 * i + j) * T + t);
    const double k = K.scale * __ldg(vol + t);
    // F = Ds Dm^-1
    double F[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const double d0 = X[1][r] - X[0][r], d1 = X[2][r] - X[0][r], d2 = X[3][r] - X[0][r];
#pragma unroll
        for (int c = 0; c < 3; ++c) F[r][c] = d0 * Dmi[0][c] + d1 * Dmi[1][c] + d2 * Dmi[2][c];
    }
    double I2 = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) I2 += F[r][c] * F[r][c];
    double cof[3][3];  // cofactor matrix dJ/dF
    {
        double c0[3] = {F[0][0], F[1][0], F[2][0]}, c1[3] = {F[0][1], F[1][1], F[2][1]},
               c2[3] = {F[0][2], F[1][2], F[2][2]}, t0[3], t1[3], t2[3];
        cross(c1, c2, t0);
        cross(c2, c0, t1);
        cross(c0, c1, t2);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            cof[r][0] = t0[r];
            cof[r][1] = t1[r];
            cof[r][2] = t2[r];
        }
    }
    const double J = F[0][0] * cof[0][0] + F[1][0] * cof[1][0] + F[2][0] * cof[2][0];
    const double Jm = J - K.alpha;
    if (energy) energy[t] = k * (0.5 * K.mu * (I2 - 3.0) + 0.5 * K.lam * Jm * Jm - 0.5 * K.mu * log(I2 + 1.0));
    if (!grad && !hess) return;   // (the line search's energy-only evaluations end here)
    const double ip1 = 1.0 / (I2 + 1.0);
    const double m1 = K.mu * (1.0 - ip1);
    if (grad) {
        // P = m1 F + lam (J - alpha) cof
        double Pm[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Pm[r][c] = m1 * F[r][c] + K.lam * Jm * cof[r][c];
        double g[12];
        map_to_x(Pm, Dmi, g);
#pragma unroll
        for (int j = 0; j < 12; ++j) grad[j * T + t] = k * g[j];
    }
    if (!hess) return;

    // the projected Hessian in the stored precision (the same operations as float64 when it is)
    using CT = HT;
    CT Fc[3][3], Dc[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            Fc[i][j] = (CT)F[i][j];
            Dc[i][j] = (CT)Dmi[i][j];
        }
    const CT m1c = (CT)m1, lJ = (CT)(K.lam * Jm), muc = (CT)K.mu, lamc = (CT)K.lam, alc = (CT)K.alpha;
    CT U[3][3], sv[3], V[3][3];
    svd3(Fc, U, sv, V);
    // Vertex blocks in the singular basis.  Mode m (F-space direction U D_m V^T) puts U D_m z_a on
    // vertex a+1 (a = 0..2), z_a = V^T (row a of Dm^-1), and minus their sum on vertex 0, so the
    // block of vertices a+1, b+1 is U M_ab U^T with M_ab = sum_m l_m+ D_m z_a z_b^T D_m^T.  With
    // twist D = (e_i e_j^T - e_j e_i^T) / sqrt2, flip D = (e_i e_j^T + e_j e_i^T) / sqrt2 (pair i < j,
    // k the third index) and the scaling modes D = diag(alpha_m):
    //   M_ab[i][i] = Ah_ii za_i zb_i + sum_{j != i} sig_k(i,j) za_j zb_j
    //   M_ab[i][j] = Ah_ij za_i zb_j + del_k(i,j) za_j zb_i                 (i != j)
    // where sig_k = (lt+ + lf+) / 2, del_k = (lf+ - lt+) / 2 and Ah = sum_m l_m+ alpha_m alpha_m^T is
    // the projected 3x3 scaling block.  Only the blocks of vertices 1..3 are formed (the diagonal
    // ones as their 6 upper entries); those of vertex 0 follow from them at the end
    // (H_0b = -sum_a H_ab, H_00 = -sum_b H_0b).
    CT z[3][3];   // z[a][i] = (V^T Dm^-T e_a)_i
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) z[a][i] = V[0][i] * Dc[a][0] + V[1][i] * Dc[a][1] + V[2][i] * Dc[a][2];
    CT sg[3], dl[3];   // per pair, indexed by its third index k
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const CT lt = CT(0.5) * (m1c + lJ * sv[k]), lf = CT(0.5) * (m1c - lJ * sv[k]);
        const CT pt = lt > CT(0) ? lt : CT(0), pf = lf > CT(0) ? lf : CT(0);
        sg[k] = pt + pf;
        dl[k] = pf - pt;
    }
    // the scaling block A = d2 Psi / ds ds and its projection Ah
    CT Ah[3][3];
    {
        CT A[3][3];
        const CT ip2 = (CT)(ip1 * ip1);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int j = (i + 1) % 3, l = (i + 2) % 3;
            A[i][i] = m1c + CT(2) * muc * sv[i] * sv[i] * ip2 + lamc * (sv[j] * sv[l]) * (sv[j] * sv[l]);
        }
        const CT sj = sv[0] * sv[1] * sv[2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i + 1; j < 3; ++j) {
                const int l = 3 - i - j;
                A[i][j] = A[j][i] = CT(2) * muc * sv[i] * sv[j] * ip2 + lamc * sv[l] * (CT(2) * sj - alc);
            }
        // Positive definite (the common case; A = L D L^T with D > 0 exists, unit lower L, no
        // pivoting): the projection is A itself.  Otherwise the eigenpairs from the Jacobi
        // iteration, the negative ones dropped.
        bool pd = A[0][0] > CT(0);
        if (pd) {
            const CT l10 = A[1][0] / A[0][0];
            const CT d1 = A[1][1] - l10 * A[1][0];
            pd = d1 > CT(0) && (A[2][2] - A[2][0] * (A[2][0] / A[0][0])) -
                                       (A[2][1] - l10 * A[2][0]) * ((A[2][1] - l10 * A[2][0]) / d1) > CT(0);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Ah[i][j] = A[i][j];
        if (!pd) {
            CT Avec[3][3];
            jacobi3(A, Avec);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j) {
                    CT h = CT(0);
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        if (A[m][m] > CT(0)) h += A[m][m] * (Avec[i][m] * Avec[j][m]);
                    Ah[i][j] = Ah[j][i] = h;
                }
        }
    }
    // the element's factor scale * vol, taken into the weights (every block is linear in them)
    {
        const CT kc = (CT)k;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            sg[i] *= kc;
            dl[i] *= kc;
#pragma unroll
            for (int j = 0; j < 3; ++j) Ah[i][j] *= kc;
        }
    }
    // M_ab, then U M_ab U^T
    auto m_ab = [&](int a, int b, CT (&M)[3][3]) {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (i == j) {
                    const int j1 = (i + 1) % 3, j2 = (i + 2) % 3;   // the pairs (i, j1), (i, j2): third index j2, j1
                    M[i][i] = Ah[i][i] * (z[a][i] * z[b][i]) + sg[j2] * (z[a][j1] * z[b][j1]) + sg[j1] * (z[a][j2] * z[b][j2]);
                } else {
                    M[i][j] = Ah[i][j] * (z[a][i] * z[b][j]) + dl[3 - i - j] * (z[a][j] * z[b][i]);
                }
            }
    };
    CT Bd[3][6], Bo[3][9];   // blocks (a,a) upper entries; blocks (0,1), (0,2), (1,2)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        CT M[3][3], T[3][3];
        m_ab(a, a, M);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) T[r][j] = U[r][0] * M[0][j] + U[r][1] * M[1][j] + U[r][2] * M[2][j];
        int e = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = r; c < 3; ++c) Bd[a][e++] = T[r][0] * U[c][0] + T[r][1] * U[c][1] + T[r][2] * U[c][2];
    }
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        const int a = o == 2 ? 1 : 0, b = o == 0 ? 1 : 2;
        CT M[3][3], T[3][3];
        m_ab(a, b, M);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) T[r][j] = U[r][0] * M[0][j] + U[r][1] * M[1][j] + U[r][2] * M[2][j];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Bo[o][3 * r + c] = T[r][0] * U[c][0] + T[r][1] * U[c][1] + T[r][2] * U[c][2];
    }
    // block (va, vb) entry (r, c) of the 12 x 12 matrix, vertices 0..3
    auto blk = [&](int a, int b, int r, int c) -> CT {   // vertices 1..3 as a, b = 0..2
        if (a == b) {
            const int lo = r < c ? r : c, hi = r < c ? c : r;
            return Bd[a][lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)];
        }
        const int o = (a + b) - 1;   // (0,1) -> 0, (0,2) -> 1, (1,2) -> 2
        return a < b ? Bo[o][3 * r + c] : Bo[o][3 * c + r];
    };
    CT H0[3][9];   // H_0b, b = vertex 1..3
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) H0[b][3 * r + c] = -((blk(0, b, r, c) + blk(1, b, r, c)) + blk(2, b, r, c));
    auto hval = [&](int p, int q) -> CT {   // H(p, q), p >= q
        const int va = p / 3, vb = q / 3, r = p % 3, c = q % 3;
        if (va == 0 && vb == 0) return -((H0[0][3 * r + c] + H0[1][3 * r + c]) + H0[2][3 * r + c]);
        if (vb == 0) return H0[va - 1][3 * c + r];   // H_a0 = H_0a^T
        if (va == 0) return H0[vb - 1][3 * r + c];
        return blk(va - 1, vb - 1, r, c);
    };
    // entry (a, b) at base + slot(a, b) * stride: element-major 3x3 sub-blocks (slot = its place
    // among the element's 144 values, stride 1) or entry-major (slot = 12 a + b, stride T)
    HT* const base = blocks ? hess + t * 144 : hess + t;
    const int64_t stride = blocks ? 1 : T;
#pragma unroll
    for (int a = 0; a < 12; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            const HT h = hval(a, b);
            const int sab = blocks ? ((a / 3) * 4 + b / 3) * 9 + (a % 3) * 3 + b % 3 : a * 12 + b;
            base[sab * stride] = h;
            if (a != b) {
                const int sba = blocks ? ((b / 3) * 4 + a / 3) * 9 + (b % 3) * 3 + a % 3 : b * 12 + a;
                base[sba * stride] = h;
            }
        }
}

// Rest state: Dm^-1 (row-major, entry-major [9][T]) and volume |det Dm| / 6.
__global__ void tet_rest_kernel(const double* __restrict__ x, int64_t n, const int32_t* __restrict__ tets,
                                int64_t T, double* __restrict__ Dm_inv, double* __restrict__ vol,
                                int32_t* __restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int32_t v[4];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        v[a] = tets[a * T + t];
        if (v[a] < 0 || v[a] >= n) ok = false;
    }
    double m[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    if (ok) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) m[r][c] = x[r * n + v[c + 1]] - x[r * n + v[0]];
    }
    const double A = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    const double B = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    const double C = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    const double det = m[0][0] * A + m[0][1] * B + m[0][2] * C;
    if (!ok || det == 0.0 || !isfinite(det)) {
        atomicAdd(bad, 1);
#pragma unroll
        for (int q = 0; q < 9; ++q) Dm_inv[q * T + t] = 0.0;
        vol[t] = 0.0;
        return;
    }
    const double id = 1.0 / det;
    const double inv[9] = {A * id, (m[0][2] * m[2][1] - m[0][1] * m[2][2]) * id, (m[0][1] * m[1][2] - m[0][2] * m[1][1]) * id,
                           B * id, (m[0][0] * m[2][2] - m[0][2] * m[2][0]) * id, (m[0][2] * m[1][0] - m[0][0] * m[1][2]) * id,
                           C * id, (m[0][1] * m[2][0] - m[0][0] * m[2][1]) * id, (m[0][0] * m[1][1] - m[0][1] * m[1][0]) * id};
#pragma unroll
    for (int q = 0; q < 9; ++q) Dm_inv[q * T + t] = inv[q];
    vol[t] = fabs(det) / 6.0;
}

// Lumped mass, deterministic: incident tetrahedra of each vertex are collected, sorted by
// index and summed in that order (density * vol / 4 each).
__global__ void mass_count_kernel(const int32_t* __restrict__ tets, int64_t T, int64_t n, int32_t* __restrict__ cnt) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int32_t v = tets[a * T + t];
        if (v >= 0 && v < n) atomicAdd(cnt + v, 1);
    }
}

__global__ void mass_fill_kernel(const int32_t* __restrict__ tets, int64_t T, int64_t n, const int64_t* __restrict__ start,
                                 unsigned long long* __restrict__ cursor, int32_t* __restrict__ list) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int32_t v = tets[a * T + t];
        if (v >= 0 && v < n) list[start[v] + (int64_t)atomicAdd(cursor + v, 1ull)] = (int32_t)t;
    }
}

__global__ void mass_sum_kernel(const int64_t* __restrict__ start, int32_t* __restrict__ list, const double* __restrict__ vol,
                                double density, int64_t n, double* __restrict__ mass) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int64_t s0 = start[v], s1 = start[v + 1];
    for (int64_t i = s0 + 1; i < s1; ++i) {  // insertion sort of the (short) incidence list
        const int32_t key = list[i];
        int64_t j = i - 1;
        while (j >= s0 && list[j] > key) {
            list[j + 1] = list[j];
            --j;
        }
        list[j + 1] = key;
    }
    double m = 0.0;
    for (int64_t i = s0; i < s1; ++i) m = __dadd_rn(m, __ddiv_rn(__dmul_rn(density, vol[list[i]]), 4.0));
    mass[v] = m;
}

__global__ void zero_cursor_kernel(unsigned long long* __restrict__ c, int32_t* __restrict__ cnt, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        c[i] = 0ull;
        cnt[i] = 0;
    }
}

inline unsigned nb(int64_t w, int t) { return (unsigned)((w + t - 1) / t); }

}  // namespace
}  // namespace gipc

extern "C" gipc_status gipc_snh_params(double young, double poisson, double* mu_h, double* lambda_h) {
    if (!mu_h || !lambda_h || !(young > 0.0) || !(poisson > -1.0 && poisson < 0.5))
        return gipc::fail(GIPC_ERR_INVALID_ARG, "gipc_snh_params: need E > 0, -1 < nu < 0.5 and outputs");
    const double mu_l = young / (2.0 * (1.0 + poisson));
    const double lam_l = young * poisson / ((1.0 + poisson) * (1.0 - 2.0 * poisson));
    *mu_h = 4.0 / 3.0 * mu_l;
    *lambda_h = lam_l + 5.0 / 6.0 * mu_l;
    return GIPC_OK;
}

extern "C" gipc_status gipc_tet_rest(gipc_ctx* ctx, const double* rest_x, int64_t n, const int32_t* tets, int64_t T,
                                     double density, double* Dm_inv, double* vol, double* mass, void* stream) {
    using namespace gipc;
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 0 || T < 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_tet_rest: negative size");
    if (mass && (!ctx || !(density > 0.0))) return fail(GIPC_ERR_INVALID_ARG, "gipc_tet_rest: mass needs a context and density > 0");
    if (T > 0 && (!rest_x || !tets || !Dm_inv || !vol)) return fail(GIPC_ERR_INVALID_ARG, "gipc_tet_rest: null pointer");
    gipc_status s;
    if (!ctx && T > 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_tet_rest: null context");
    if (T > 0) {
        if ((s = ctx->slot[0].reserve(sizeof(int32_t) * 4)) != GIPC_OK) return s;
        int32_t* bad = ctx->slot[0].as<int32_t>();
        cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
        tet_rest_kernel<<<nb(T, 128), 128, 0, st>>>(rest_x, n, tets, T, Dm_inv, vol, bad);
        int32_t hbad = 0;
        cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_tet_rest");
        if (hbad) return fail(GIPC_ERR_INVALID_ARG, "gipc_tet_rest: %d degenerate or out-of-range tetrahedra", hbad);
    }
    if (mass && n > 0) {
        const int64_t links = 4 * T;
        if ((s = ctx->slot[1].reserve(sizeof(int32_t) * (n + 1) + 16)) != GIPC_OK) return s;
        if ((s = ctx->slot[2].reserve(sizeof(int64_t) * (n + 2 + scan_scratch_words(n + 1)) + sizeof(unsigned long long) * n)) != GIPC_OK) return s;
        if ((s = ctx->slot[3].reserve(sizeof(int32_t) * (links + 1))) != GIPC_OK) return s;
        int32_t* cnt = ctx->slot[1].as<int32_t>();
        int64_t* start = ctx->slot[2].as<int64_t>();
        int64_t* scan_tmp = start + n + 2;
        unsigned long long* cursor = reinterpret_cast<unsigned long long*>(scan_tmp + scan_scratch_words(n + 1));
        int32_t* list = ctx->slot[3].as<int32_t>();
        zero_cursor_kernel<<<nb(n, 256), 256, 0, st>>>(cursor, cnt, n);
        if (T > 0) mass_count_kernel<<<nb(T, 256), 256, 0, st>>>(tets, T, n, cnt);
        if (exclusive_scan<int32_t>(cnt, start, n, scan_tmp, st) != cudaSuccess) return check_launch("gipc_tet_rest: scan");
        if (T > 0) mass_fill_kernel<<<nb(T, 256), 256, 0, st>>>(tets, T, n, start, cursor, list);
        mass_sum_kernel<<<nb(n, 256), 256, 0, st>>>(start, list, vol, density, n, mass);
    }
    return check_launch("gipc_tet_rest");
}

namespace gipc {
// gipc_eval_tets, the elements of the scenes s with live[s] == 0 (vscene: the scene of every
// vertex) left out with zero outputs; live == NULL evaluates every element.
gipc_status eval_tets_live(const double* x, int64_t n, const int32_t* tets, int64_t T, const double* Dm_inv,
                           const double* vol, const gipc_elastic_params* prm, int prec, int hess_mode, double* energy,
                           double* grad, void* hess, const int32_t* vscene, const int32_t* live, cudaStream_t stream) {
    if (n < 0 || T < 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_tets: negative size");
    if (!prm || !(prm->mu > 0.0) || !(prm->lambda > 0.0) || !(prm->scale >= 0.0))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_tets: need mu > 0, lambda > 0, scale >= 0");
    if (prec != GIPC_FP64 && prec != GIPC_MIXED) return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_tets: bad precision");
    if (hess_mode != GIPC_HESS_DENSE && hess_mode != GIPC_HESS_BLOCKS)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_tets: hess_mode must be GIPC_HESS_DENSE or GIPC_HESS_BLOCKS");
    if (T == 0) return GIPC_OK;
    if (!x || !tets || !Dm_inv || !vol) return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_tets: null input");
    ElasticConst K{prm->mu, prm->lambda, 1.0 + prm->mu / prm->lambda - prm->mu / (4.0 * prm->lambda), prm->scale};
    cudaStream_t st = stream;
    const bool blk = hess_mode == GIPC_HESS_BLOCKS;
    if (live && !vscene) return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_tets: scene mask without the vertex scenes");
    if (prec == GIPC_FP64)
        eval_tets_kernel<GIPC_FP64><<<nb(T, 128), 128, 0, st>>>(x, n, tets, T, Dm_inv, vol, K, energy, grad, hess, blk,
                                                                 vscene, live);
    else
        eval_tets_kernel<GIPC_MIXED><<<nb(T, 128), 128, 0, st>>>(x, n, tets, T, Dm_inv, vol, K, energy, grad, hess, blk,
                                                                  vscene, live);
    return check_launch("gipc_eval_tets");
}
}  // namespace gipc

extern "C" gipc_status gipc_eval_tets(const double* x, int64_t n, const int32_t* tets, int64_t T, const double* Dm_inv,
                                      const double* vol, const gipc_elastic_params* prm, int prec, int hess_mode,
                                      double* energy, double* grad, void* hess, void* stream) {
    return gipc::eval_tets_live(x, n, tets, T, Dm_inv, vol, prm, prec, hess_mode, energy, grad, hess, nullptr, nullptr,
                                (cudaStream_t)stream);
}
