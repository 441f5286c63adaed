/*
 * FP64 reference state-vector simulator -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the oracle that the CUDA library is checked against.  It is
 * written for a reader who wants to compare it with the paper by eye: every
 * gate is applied with a plain loop over the whole amplitude array, Pauli
 * strings are applied factor by factor to a copy, and gradients come from the
 * textbook adjoint sweep.  There is no blocking, fusion or reordering.  Only
 * tests, the package smoke check and the benchmark's CPU-baseline leg may
 * load it; the product path never does.
 *
 * Passages followed (DeepQuantum, arXiv 2512.18995):
 *   - Sec. "Quantum Computing with Qubits", Background: single-qubit basis
 *     |0>, |1> as Z eigenstates and the Bloch form cos(t/2)|0> +
 *     e^{i p} sin(t/2)|1>, and the evolution |psi_n> = U_n ... U_1 |psi_0>.
 *   - Same section, API Overview: circuits built by appending gates, forward
 *     execution, expectation values of observables given as Pauli strings.
 *   - Sec. "Large-Scale Simulations", Distributed Simulations: gradients of
 *     expectations with respect to trainable parameters and encoded inputs by
 *     the adjoint differentiation method (Jones & Gacon, arXiv:2009.02823).
 *   - Sec. "Simulation of Large Quantum Systems with MPS" (Trotterised TFIM
 *     with rx(-h dt), rzz(-2 J dt)): rotations are R_P(t) = exp(-i t P / 2).
 *   - Sec. "Distributed Quantum Fourier Transform": controlled phase
 *     CP(phi) = diag(1, 1, 1, e^{i phi}), Hadamard, SWAP.
 *   - Sec. "Quantum Machine Learning" (QNN, QCNN examples) and the Trotterised
 *     TFIM: the general one-qubit gate u3, the two-qubit rotations rxx, ryy,
 *     rzz (R_PP(t) = exp(-i t P(x)P / 2), the same exp(-i t G / 2) form),
 *     controlled RY with an encoded angle.  The phase shift P(t) = diag(1,
 *     e^{it}) and the Toffoli gate CCX complete the gate set.
 *   - Dense blocks (oracle_apply_dense): the same evolution with a group of
 *     consecutive gates written as one matrix on the lowest-order wires; the
 *     paper applies gates one at a time, so this is the plain definition of
 *     a matrix acting on a subset of wires.
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   - wire 0 is the most significant bit of the amplitude index:
 *       index = sum_q b_q 2^(n-1-q).
 *   - RZ(t) = diag(e^{-i t/2}, e^{i t/2}) (the exp(-i t Z / 2) form).
 *   - a Pauli term carries bit q of xmask/zmask for wire q; both bits = Y.
 *   - U3(theta, phi, lam) = [[cos(theta/2), -e^{i lam} sin(theta/2)],
 *     [e^{i phi} sin(theta/2), e^{i(phi+lam)} cos(theta/2)]] (the usual u3
 *     matrix; its first column is the Bloch form of the Background section),
 *     with its three angles in consecutive parameter (or feature) slots.
 *
 * Parity: pinned (closed forms, brute-force dense products, parameter-shift
 * and finite differences in the test-suite).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Gate codes of the oracle (independent of the library's own enum). */
enum {
    O_H = 0, O_X, O_Y, O_Z, O_S,
    O_RX, O_RY, O_RZ,
    O_CNOT, O_CZ, O_CP, O_SWAP,
    O_CRX, O_CRY, O_CRZ,
    O_P, O_U3, O_RXX, O_RYY, O_RZZ, O_CCX,
    O_BITFLIP, O_PHASEFLIP, O_DEPOLARIZING, O_AMPDAMP,
    O_NKINDS
};

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gate matrices.                                                             */
/* ------------------------------------------------------------------------ */

/* 2x2 matrix m = [[m0, m1], [m2, m3]] acting on the target qubit.  For a
 * controlled gate this is the block applied when the control is |1>.
 * Rotations follow R_P(t) = cos(t/2) I - i sin(t/2) P, which is exp(-i t P/2)
 * because P^2 = I. */
static void target_matrix(int kind, double t, cplx m[4])
{
    const double c = cos(0.5 * t), s = sin(0.5 * t);
    const double r = 1.0 / sqrt(2.0);
    switch (kind) {
    case O_H:    m[0] = r;  m[1] = r;   m[2] = r;  m[3] = -r;  break;
    case O_X:
    case O_CNOT: m[0] = 0;  m[1] = 1;   m[2] = 1;  m[3] = 0;   break;
    case O_Y:    m[0] = 0;  m[1] = -I;  m[2] = I;  m[3] = 0;   break;
    case O_Z:
    case O_CZ:   m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = -1;  break;
    case O_S:    m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = I;   break;
    case O_RX:
    case O_CRX:  m[0] = c;  m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    case O_RY:
    case O_CRY:  m[0] = c;  m[1] = -s;  m[2] = s;  m[3] = c;   break;
    case O_RZ:
    case O_CRZ:  m[0] = c - I * s; m[1] = 0; m[2] = 0; m[3] = c + I * s; break;
    case O_CP:   m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = cexp(I * t); break;
    case O_P:    m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = cexp(I * t); break;
    default:     m[0] = 1;  m[1] = 0;   m[2] = 0;  m[3] = 1;   break;
    }
}

/* Generator G with U(t) = exp(-i t G) for the parametric gates, as a 2x2
 * block on the target (restricted to the control = |1> subspace for
 * controlled gates).  d/dt U = -i G U. */
static void generator_matrix(int kind, cplx g[4])
{
    g[0] = g[1] = g[2] = g[3] = 0;
    switch (kind) {
    case O_RX: case O_CRX: g[1] = 0.5;       g[2] = 0.5;      break;  /* X/2 */
    case O_RY: case O_CRY: g[1] = -0.5 * I;  g[2] = 0.5 * I;  break;  /* Y/2 */
    case O_RZ: case O_CRZ: g[0] = 0.5;       g[3] = -0.5;     break;  /* Z/2 */
    case O_CP:             g[3] = -1.0;                        break;  /* CP = exp(i t |11><11|) */
    case O_P:              g[3] = -1.0;                        break;  /* P = exp(i t |1><1|) */
    default: break;
    }
}

static int is_parametric(int kind)
{
    return kind == O_RX || kind == O_RY || kind == O_RZ || kind == O_CP ||
           kind == O_CRX || kind == O_CRY || kind == O_CRZ || kind == O_P ||
           kind == O_U3 || kind == O_RXX || kind == O_RYY || kind == O_RZZ;
}

/* Number of consecutive angle slots a gate reads (U3: theta, phi, lam). */
static int angle_span(int kind) { return kind == O_U3 ? 3 : 1; }

/* U3(theta, phi, lam) and its partial derivatives, written out from the
 * matrix definition:
 *   U  = [[ch, -e^{i lam} sh], [e^{i phi} sh, e^{i(phi+lam)} ch]]
 *   dU/dtheta = 1/2 [[-sh, -e^{i lam} ch], [e^{i phi} ch, -e^{i(phi+lam)} sh]]
 *   dU/dphi   = [[0, 0], [i e^{i phi} sh, i e^{i(phi+lam)} ch]]
 *   dU/dlam   = [[0, -i e^{i lam} sh], [0, i e^{i(phi+lam)} ch]]
 * with ch = cos(theta/2), sh = sin(theta/2).  which = 0 gives U, 1..3 the
 * derivative in theta, phi, lam. */
static void u3_matrix(const double t3[3], int which, cplx m[4])
{
    const double ch = cos(t3[0] / 2.0), sh = sin(t3[0] / 2.0);
    const cplx ep = cexp(I * t3[1]), el = cexp(I * t3[2]), epl = cexp(I * (t3[1] + t3[2]));
    switch (which) {
    case 0: m[0] = ch;        m[1] = -el * sh;      m[2] = ep * sh;      m[3] = epl * ch;       break;
    case 1: m[0] = -0.5 * sh; m[1] = -0.5 * el * ch; m[2] = 0.5 * ep * ch; m[3] = -0.5 * epl * sh; break;
    case 2: m[0] = 0;         m[1] = 0;             m[2] = I * ep * sh;  m[3] = I * epl * ch;   break;
    default: m[0] = 0;        m[1] = -I * el * sh;  m[2] = 0;            m[3] = I * epl * ch;   break;
    }
}

static int is_controlled(int kind)
{
    return kind == O_CNOT || kind == O_CZ || kind == O_CP ||
           kind == O_CRX || kind == O_CRY || kind == O_CRZ;
}

static int is_pauli_pair(int kind) { return kind == O_RXX || kind == O_RYY || kind == O_RZZ; }

/* Bit position of wire q: wire 0 is the most significant bit. */
static inline int bitpos(int n, int q) { return n - 1 - q; }

/* ------------------------------------------------------------------------ */
/* Plain per-gate application over the whole array.                          */
/* ------------------------------------------------------------------------ */

/* Apply 2x2 block m to the target wire, on the amplitudes whose control wire
 * is |1> (ctrl < 0: no control). */
static void apply_block(int n, cplx *psi, int target, int ctrl, const cplx m[4])
{
    const int64_t dim = (int64_t)1 << n;
    const int64_t tb = (int64_t)1 << bitpos(n, target);
    const int64_t cb = ctrl >= 0 ? ((int64_t)1 << bitpos(n, ctrl)) : 0;
#pragma omp parallel for schedule(static) if (dim >= (1 << 16))
    for (int64_t i = 0; i < dim; ++i) {
        if (i & tb) continue;                 /* visit each pair once */
        if (cb && !(i & cb)) continue;        /* control must be |1> */
        const int64_t j = i | tb;
        const cplx a = psi[i], b = psi[j];
        psi[i] = m[0] * a + m[1] * b;
        psi[j] = m[2] * a + m[3] * b;
    }
}

static void apply_swap(int n, cplx *psi, int qa, int qb)
{
    const int64_t dim = (int64_t)1 << n;
    const int64_t ba = (int64_t)1 << bitpos(n, qa);
    const int64_t bb = (int64_t)1 << bitpos(n, qb);
#pragma omp parallel for schedule(static) if (dim >= (1 << 16))
    for (int64_t i = 0; i < dim; ++i) {
        if ((i & ba) && !(i & bb)) {          /* |..1..0..> <-> |..0..1..> */
            const int64_t j = (i & ~ba) | bb;
            const cplx t = psi[i];
            psi[i] = psi[j];
            psi[j] = t;
        }
    }
}

/* Apply X on the target wire of the amplitudes whose two control wires are
 * both |1> (Toffoli). */
static void apply_ccx(int n, cplx *psi, int c0, int c1, int target)
{
    const int64_t dim = (int64_t)1 << n;
    const int64_t b0 = (int64_t)1 << bitpos(n, c0);
    const int64_t b1 = (int64_t)1 << bitpos(n, c1);
    const int64_t tb = (int64_t)1 << bitpos(n, target);
#pragma omp parallel for schedule(static) if (dim >= (1 << 16))
    for (int64_t i = 0; i < dim; ++i) {
        if ((i & tb) || !(i & b0) || !(i & b1)) continue;
        const int64_t j = i | tb;
        const cplx a = psi[i];
        psi[i] = psi[j];
        psi[j] = a;
    }
}

/* Apply one Pauli string (masks by wire) factor by factor. */
static void apply_pauli(int n, cplx *v, uint64_t xmask, uint64_t zmask)
{
    for (int q = 0; q < n; ++q) {
        const int x = (int)((xmask >> q) & 1), z = (int)((zmask >> q) & 1);
        if (!x && !z) continue;
        const int kind = (x && z) ? O_Y : (x ? O_X : O_Z);
        cplx m[4];
        target_matrix(kind, 0.0, m);
        apply_block(n, v, q, -1, m);
    }
}

/* The two-qubit Pauli string P(x)P of kind RXX / RYY / RZZ on wires a, b, as
 * (xmask, zmask) by wire. */
static void pauli_pair_masks(int kind, int a, int b, uint64_t *xm, uint64_t *zm)
{
    const uint64_t w = ((uint64_t)1 << a) | ((uint64_t)1 << b);
    *xm = (kind == O_RXX || kind == O_RYY) ? w : 0;
    *zm = (kind == O_RZZ || kind == O_RYY) ? w : 0;
}

/* psi <- exp(-i t S / 2) psi = cos(t/2) psi - i sin(t/2) S psi for a Pauli
 * string S (S^2 = I), with S psi formed on a copy. */
static void apply_pauli_rotation(int n, cplx *psi, uint64_t xm, uint64_t zm, double t)
{
    const int64_t dim = (int64_t)1 << n;
    cplx *sp = (cplx *)malloc((size_t)dim * sizeof(cplx));
    memcpy(sp, psi, (size_t)dim * sizeof(cplx));
    apply_pauli(n, sp, xm, zm);
    const double c = cos(t / 2.0), sn = sin(t / 2.0);
    for (int64_t i = 0; i < dim; ++i) psi[i] = c * psi[i] - I * sn * sp[i];
    free(sp);
}

/* Angles of gate g for batch row `row`: t3[k] for k < angle_span(kind),
 * from consecutive parameter or feature slots, else the fixed angle. */
static void gate_angles(int g, int kind, const int *pidx, const int *didx, const double *angle,
                        const double *params, int nparams, int params_per_row,
                        const double *data, int nfeat, int row, double t3[3])
{
    t3[0] = t3[1] = t3[2] = 0.0;
    for (int k = 0; k < angle_span(kind); ++k) {
        if (pidx[g] >= 0)
            t3[k] = params_per_row ? params[(int64_t)row * nparams + pidx[g] + k] : params[pidx[g] + k];
        else if (didx[g] >= 0)
            t3[k] = data[(int64_t)row * nfeat + didx[g] + k];
        else
            t3[k] = angle[g];
    }
}

static void conj_transpose(const cplx m[4], cplx d[4])
{
    d[0] = conj(m[0]); d[1] = conj(m[2]); d[2] = conj(m[1]); d[3] = conj(m[3]);
}

/* Apply gate g (or its inverse when `dagger`); t3 holds its angles. */
static void apply_gate(int n, cplx *psi, int kind, int w0, int w1, int w2, const double t3[3], int dagger)
{
    if (kind == O_SWAP) {
        apply_swap(n, psi, w0, w1);
        return;
    }
    if (kind == O_CCX) {
        apply_ccx(n, psi, w0, w1, w2);
        return;
    }
    if (is_pauli_pair(kind)) {
        uint64_t xm, zm;
        pauli_pair_masks(kind, w0, w1, &xm, &zm);
        apply_pauli_rotation(n, psi, xm, zm, dagger ? -t3[0] : t3[0]);
        return;
    }
    cplx m[4], d[4];
    if (kind == O_U3)
        u3_matrix(t3, 0, m);
    else
        target_matrix(kind, t3[0], m);
    if (dagger) {
        conj_transpose(m, d);
        memcpy(m, d, sizeof(m));
    }
    if (is_controlled(kind))
        apply_block(n, psi, w1, w0, m);
    else
        apply_block(n, psi, w0, -1, m);
}

/* Single-row forward run from |0...0>. */
static void run_row(int n, int ngates, const int *kind, const int *w0, const int *w1, const int *w2,
                    const int *pidx, const int *didx, const double *angle,
                    const double *params, int nparams, int params_per_row,
                    const double *data, int nfeat, int row, cplx *psi)
{
    const int64_t dim = (int64_t)1 << n;
    for (int64_t i = 0; i < dim; ++i) psi[i] = 0;
    psi[0] = 1;
    for (int g = 0; g < ngates; ++g) {
        double t3[3];
        gate_angles(g, kind[g], pidx, didx, angle, params, nparams, params_per_row, data, nfeat, row, t3);
        apply_gate(n, psi, kind[g], w0[g], w1[g], w2[g], t3, 0);
    }
}

static cplx inner(int64_t dim, const cplx *a, const cplx *b)  /* <a|b> */
{
    cplx s = 0;
    for (int64_t i = 0; i < dim; ++i) s += conj(a[i]) * b[i];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Exported API.                                                              */
/* ------------------------------------------------------------------------ */

/* Gate matrix for checking against independent definitions (2x2 target block
 * for one-qubit and controlled kinds). */
void oracle_gate_block(int kind, double t, double *out8)
{
    cplx m[4];
    target_matrix(kind, t, m);
    for (int i = 0; i < 4; ++i) { out8[2 * i] = creal(m[i]); out8[2 * i + 1] = cimag(m[i]); }
}

/* Apply a gate list to `batch` given states in place (used for unitarity and
 * dense-matrix checks, where the input is not |0...0>). */
void oracle_apply(int n, int ngates, const int *kind, const int *w0, const int *w1, const int *w2,
                  const int *pidx, const int *didx, const double *angle,
                  const double *params, int nparams, int params_per_row,
                  const double *data, int nfeat, int batch, int dagger, double *states_ri)
{
    const int64_t dim = (int64_t)1 << n;
    cplx *states = (cplx *)states_ri;
#pragma omp parallel for schedule(dynamic, 1) if (batch > 1)
    for (int r = 0; r < batch; ++r) {
        cplx *psi = states + (int64_t)r * dim;
        for (int step = 0; step < ngates; ++step) {
            const int g = dagger ? ngates - 1 - step : step;
            double t3[3];
            gate_angles(g, kind[g], pidx, didx, angle, params, nparams, params_per_row, data, nfeat, r, t3);
            apply_gate(n, psi, kind[g], w0[g], w1[g], w2[g], t3, dagger);
        }
    }
}

/* |psi_row> = U_G ... U_1 |0...0> for every batch row. */
void oracle_run(int n, int ngates, const int *kind, const int *w0, const int *w1, const int *w2,
                const int *pidx, const int *didx, const double *angle,
                const double *params, int nparams, int params_per_row,
                const double *data, int nfeat, int batch, double *states_ri)
{
    const int64_t dim = (int64_t)1 << n;
    cplx *states = (cplx *)states_ri;
#pragma omp parallel for schedule(dynamic, 1) if (batch > 1)
    for (int r = 0; r < batch; ++r)
        run_row(n, ngates, kind, w0, w1, w2, pidx, didx, angle, params, nparams,
                params_per_row, data, nfeat, r, states + (int64_t)r * dim);
}

/* out[row*nobs + o] = sum_{k in obs o} coeff_k Re <psi_row| P_k |psi_row>. */
void oracle_expect(int n, const double *coeff, const uint64_t *xmask, const uint64_t *zmask,
                   const int *term_offsets, int nobs, int batch, const double *states_ri,
                   double *out)
{
    const int64_t dim = (int64_t)1 << n;
    const cplx *states = (const cplx *)states_ri;
#pragma omp parallel for schedule(dynamic, 1) if (batch > 1)
    for (int r = 0; r < batch; ++r) {
        const cplx *psi = states + (int64_t)r * dim;
        cplx *tmp = (cplx *)malloc((size_t)dim * sizeof(cplx));
        for (int o = 0; o < nobs; ++o) {
            double acc = 0.0;
            for (int k = term_offsets[o]; k < term_offsets[o + 1]; ++k) {
                memcpy(tmp, psi, (size_t)dim * sizeof(cplx));
                apply_pauli(n, tmp, xmask[k], zmask[k]);
                acc += coeff[k] * creal(inner(dim, psi, tmp));
            }
            out[(int64_t)r * nobs + o] = acc;
        }
        free(tmp);
    }
}

/*
 * Adjoint differentiation (Jones & Gacon 2020) of
 *     L = sum_row sum_o w[row, o] * E[row, o],
 * with E[row, o] = <psi_row| O_o |psi_row> and w = row_weights (NULL = 1).
 *
 *   psi <- U_G ... U_1 |0>,   lambda <- (sum_o w_o O_o) psi
 *   for j = G .. 1:
 *       if gate j has an angle t_j = exp(-i t G_j):
 *           dL/dt_j += 2 Im <lambda | G_j | psi>
 *       (U3, whose angles enter otherwise: dL/dt_k += 2 Re <lambda| dU/dt_k
 *        U^dagger psi>, the same derivative before the generator is factored)
 *       psi <- U_j^dagger psi,  lambda <- U_j^dagger lambda
 *
 * The derivative is routed to the trainable parameter (summed over rows when
 * params are shared, per row when params_per_row) or to the encoded feature
 * (per row).  expect_out (batch x nobs) receives E.
 */
void oracle_adjoint(int n, int ngates, const int *kind, const int *w0, const int *w1, const int *w2,
                    const int *pidx, const int *didx, const double *angle,
                    const double *params, int nparams, int params_per_row,
                    const double *data, int nfeat, int batch,
                    const double *coeff, const uint64_t *xmask, const uint64_t *zmask,
                    const int *term_offsets, int nobs, const double *row_weights,
                    double *expect_out, double *grad_params, double *grad_data)
{
    const int64_t dim = (int64_t)1 << n;
    const int gp_rows = params_per_row ? batch : 1;
    double *gp_row = (double *)calloc((size_t)batch * (nparams > 0 ? nparams : 1), sizeof(double));

#pragma omp parallel for schedule(dynamic, 1) if (batch > 1)
    for (int r = 0; r < batch; ++r) {
        cplx *psi = (cplx *)malloc((size_t)dim * sizeof(cplx));
        cplx *lam = (cplx *)calloc((size_t)dim, sizeof(cplx));
        cplx *tmp = (cplx *)malloc((size_t)dim * sizeof(cplx));
        cplx *tmp2 = (cplx *)malloc((size_t)dim * sizeof(cplx));
        double *gp = gp_row + (int64_t)r * (nparams > 0 ? nparams : 1);

        run_row(n, ngates, kind, w0, w1, w2, pidx, didx, angle, params, nparams,
                params_per_row, data, nfeat, r, psi);

        /* expectations and lambda = sum_o w_o O_o psi */
        for (int o = 0; o < nobs; ++o) {
            const double w = row_weights ? row_weights[(int64_t)r * nobs + o] : 1.0;
            double acc = 0.0;
            for (int k = term_offsets[o]; k < term_offsets[o + 1]; ++k) {
                memcpy(tmp, psi, (size_t)dim * sizeof(cplx));
                apply_pauli(n, tmp, xmask[k], zmask[k]);
                acc += coeff[k] * creal(inner(dim, psi, tmp));
                for (int64_t i = 0; i < dim; ++i) lam[i] += w * coeff[k] * tmp[i];
            }
            if (expect_out) expect_out[(int64_t)r * nobs + o] = acc;
        }
        if (grad_data)
            for (int f = 0; f < nfeat; ++f) grad_data[(int64_t)r * nfeat + f] = 0.0;

        for (int g = ngates - 1; g >= 0; --g) {
            double t3[3];
            gate_angles(g, kind[g], pidx, didx, angle, params, nparams, params_per_row, data, nfeat, r, t3);
            const int trainable = is_parametric(kind[g]) && (pidx[g] >= 0 || didx[g] >= 0);
            if (trainable && kind[g] == O_U3) {
                /* U3 is not of the exp(-i t G) form in each angle: take
                 * dL/dt_k = 2 Re <lambda| (dU/dt_k) psi_before> with
                 * psi_before = U^dagger psi. */
                memcpy(tmp, psi, (size_t)dim * sizeof(cplx));
                apply_gate(n, tmp, O_U3, w0[g], -1, -1, t3, 1);
                for (int k = 0; k < 3; ++k) {
                    cplx dm[4];
                    u3_matrix(t3, k + 1, dm);
                    memcpy(tmp2, tmp, (size_t)dim * sizeof(cplx));
                    apply_block(n, tmp2, w0[g], -1, dm);
                    const double dk = 2.0 * creal(inner(dim, lam, tmp2));
                    if (pidx[g] >= 0) gp[pidx[g] + k] += dk;
                    else if (grad_data) grad_data[(int64_t)r * nfeat + didx[g] + k] += dk;
                }
            } else if (trainable) {
                memcpy(tmp, psi, (size_t)dim * sizeof(cplx));
                if (is_pauli_pair(kind[g])) {
                    /* R_S(t) = exp(-i t S / 2): generator S / 2 */
                    uint64_t xm, zm;
                    pauli_pair_masks(kind[g], w0[g], w1[g], &xm, &zm);
                    apply_pauli(n, tmp, xm, zm);
                    for (int64_t i = 0; i < dim; ++i) tmp[i] *= 0.5;
                } else {
                    cplx gm[4];
                    generator_matrix(kind[g], gm);
                    if (is_controlled(kind[g])) {
                        /* generator lives on the control=|1> subspace */
                        const int64_t cb = (int64_t)1 << bitpos(n, w0[g]);
                        for (int64_t i = 0; i < dim; ++i)
                            if (!(i & cb)) tmp[i] = 0;
                        apply_block(n, tmp, w1[g], w0[g], gm);
                    } else {
                        apply_block(n, tmp, w0[g], -1, gm);
                    }
                }
                const double d = 2.0 * cimag(inner(dim, lam, tmp));
                if (pidx[g] >= 0) gp[pidx[g]] += d;
                else if (grad_data) grad_data[(int64_t)r * nfeat + didx[g]] += d;
            }
            apply_gate(n, psi, kind[g], w0[g], w1[g], w2[g], t3, 1);
            apply_gate(n, lam, kind[g], w0[g], w1[g], w2[g], t3, 1);
        }
        free(psi);
        free(lam);
        free(tmp);
        free(tmp2);
    }

    if (grad_params && nparams > 0) {
        if (params_per_row) {
            memcpy(grad_params, gp_row, (size_t)batch * nparams * sizeof(double));
        } else {
            for (int p = 0; p < nparams; ++p) {
                double s = 0.0;
                for (int r = 0; r < batch; ++r) s += gp_row[(int64_t)r * nparams + p];
                grad_params[p] = s;
            }
        }
    }
    (void)gp_rows;
    free(gp_row);
}

/* ------------------------------------------------------------------------ */
/* Hessian.                                                                  */
/* ------------------------------------------------------------------------ */

/* Second partial derivatives of U3 (which = 0, 1, 2 for theta, phi, lam),
 * from the matrix definition: every entry is a product of one of
 * cos(theta/2), sin(theta/2) with a phase e^{i(a phi + b lam)}, so each
 * derivative multiplies it by the matching factor (-sin/2 <-> cos/2 for
 * theta, i a for phi, i b for lam). */
static void u3_second(const double t3[3], int wa, int wb, cplx m[4])
{
    const double ch = cos(t3[0] / 2.0), sh = sin(t3[0] / 2.0);
    /* entry e: trig part T_e(theta) and phase exponents (a_e, b_e) */
    const double ca[4] = {0, 0, 1, 1}, cb[4] = {0, 1, 0, 1};
    const double sgn[4] = {1, -1, 1, 1};
    const int usesin[4] = {0, 1, 1, 0};
    for (int e = 0; e < 4; ++e) {
        /* trig part and its theta derivatives: f, f', f'' */
        const double f0 = usesin[e] ? sh : ch;
        const double f1 = usesin[e] ? 0.5 * ch : -0.5 * sh;
        const double f2 = -0.25 * f0;
        int nth = (wa == 0) + (wb == 0);
        const double trig = nth == 0 ? f0 : (nth == 1 ? f1 : f2);
        cplx fac = 1.0;
        if (wa == 1) fac *= I * ca[e];
        if (wa == 2) fac *= I * cb[e];
        if (wb == 1) fac *= I * ca[e];
        if (wb == 2) fac *= I * cb[e];
        m[e] = sgn[e] * trig * fac * cexp(I * (ca[e] * t3[1] + cb[e] * t3[2]));
    }
}

/* v <- G v for the generator G of gate kind (U(t) = exp(-i t G)); controlled
 * kinds: G acts on the control = |1> subspace only. */
static void apply_generator(int n, cplx *v, int kind, int w0, int w1)
{
    const int64_t dim = (int64_t)1 << n;
    if (is_pauli_pair(kind)) {
        uint64_t xm, zm;
        pauli_pair_masks(kind, w0, w1, &xm, &zm);
        apply_pauli(n, v, xm, zm);
        for (int64_t i = 0; i < dim; ++i) v[i] *= 0.5;
        return;
    }
    cplx gm[4];
    generator_matrix(kind, gm);
    if (is_controlled(kind)) {
        const int64_t cb = (int64_t)1 << bitpos(n, w0);
        for (int64_t i = 0; i < dim; ++i)
            if (!(i & cb)) v[i] = 0;
        apply_block(n, v, w1, w0, gm);
    } else {
        apply_block(n, v, w0, -1, gm);
    }
}

/* Apply gate g to v, differentiated with respect to angle slots: nd = 0
 * (the gate), 1 (d/dt_ka) or 2 (d^2/dt_ka dt_kb).  For exp(-i t G):
 * dU = -i G U, d^2U = -G^2 U; U3 uses its derivative matrices. */
static void apply_gate_diff(int n, cplx *v, int kind, int w0, int w1, int w2, const double t3[3], int nd,
                            int ka, int kb)
{
    const int64_t dim = (int64_t)1 << n;
    if (nd == 0) {
        apply_gate(n, v, kind, w0, w1, w2, t3, 0);
        return;
    }
    if (kind == O_U3) {
        cplx m[4];
        if (nd == 1) u3_matrix(t3, ka + 1, m);
        else u3_second(t3, ka, kb, m);
        apply_block(n, v, w0, -1, m);
        return;
    }
    apply_gate(n, v, kind, w0, w1, w2, t3, 0);
    apply_generator(n, v, kind, w0, w1);
    if (nd == 2) apply_generator(n, v, kind, w0, w1);
    const cplx f = nd == 1 ? -I : -1.0;
    for (int64_t i = 0; i < dim; ++i) v[i] *= f;
}

/*
 * Hessian of L = sum_row sum_o w[row, o] <psi_row| O_o |psi_row> with respect
 * to the shared trainable parameters (the second derivatives of the paper's
 * gradient-and-Hessian benchmark), by the product rule on the circuit:
 * with O = sum_o w_o O_o, psi_a the final state with occurrence a's gate
 * differentiated in its angle, and psi_ab the state with both differentiated
 * (a second derivative when a and b are angles of the same gate),
 *     d^2 L / dt_a dt_b = 2 Re( <psi_ab|O|psi> + <psi_a|O|psi_b> ).
 * An occurrence is one angle slot of one gate with a trainable parameter;
 * parameters used several times collect their occurrences' sums.
 * hess: nparams x nparams, overwritten.  Every pair costs a forward run
 * (plain and slow by construction).
 */
void oracle_hessian(int n, int ngates, const int *kind, const int *w0, const int *w1, const int *w2,
                    const int *pidx, const int *didx, const double *angle,
                    const double *params, int nparams, const double *data, int nfeat, int batch,
                    const double *coeff, const uint64_t *xmask, const uint64_t *zmask,
                    const int *term_offsets, int nobs, const double *row_weights, double *hess)
{
    const int64_t dim = (int64_t)1 << n;
    /* occurrences (gate, angle slot) */
    int nocc = 0;
    for (int g = 0; g < ngates; ++g)
        if (is_parametric(kind[g]) && pidx[g] >= 0) nocc += angle_span(kind[g]);
    int *og = (int *)malloc(sizeof(int) * (nocc + 1)), *ok = (int *)malloc(sizeof(int) * (nocc + 1));
    for (int g = 0, a = 0; g < ngates; ++g)
        if (is_parametric(kind[g]) && pidx[g] >= 0)
            for (int k = 0; k < angle_span(kind[g]); ++k, ++a) { og[a] = g; ok[a] = k; }
    double *acc = (double *)calloc((size_t)nparams * (nparams > 0 ? nparams : 1) + 1, sizeof(double));

    for (int r = 0; r < batch; ++r) {
        /* the states: psi, psi_a, and per pair psi_ab */
        cplx *psi = (cplx *)malloc((size_t)dim * sizeof(cplx));
        cplx *Opsi = (cplx *)calloc((size_t)dim, sizeof(cplx));
        cplx *tmp = (cplx *)malloc((size_t)dim * sizeof(cplx));
        cplx *pa = (cplx *)malloc((size_t)dim * (nocc + 1) * sizeof(cplx));
        cplx *Opa = (cplx *)calloc((size_t)dim * (nocc + 1), sizeof(cplx));
        /* run the circuit with occurrence sets differentiated */
        #define RUN_DIFF(out_, a_, b_)                                                                      \
            do {                                                                                           \
                for (int64_t i = 0; i < dim; ++i) (out_)[i] = 0;                                           \
                (out_)[0] = 1;                                                                             \
                for (int g = 0; g < ngates; ++g) {                                                         \
                    double t3[3];                                                                          \
                    gate_angles(g, kind[g], pidx, didx, angle, params, nparams, 0, data, nfeat, r, t3);    \
                    int nd = 0, ka = 0, kb = 0;                                                            \
                    if ((a_) >= 0 && og[(a_)] == g) { nd++; ka = ok[(a_)]; }                               \
                    if ((b_) >= 0 && og[(b_)] == g) { if (nd) kb = ok[(b_)]; else ka = ok[(b_)]; nd++; }  \
                    apply_gate_diff(n, (out_), kind[g], w0[g], w1[g], w2[g], t3, nd, ka, kb);              \
                }                                                                                          \
            } while (0)
        /* O applied to a state: sum_o w_o sum_k c_k P_k */
        #define APPLY_O(dst_, src_)                                                                        \
            do {                                                                                           \
                for (int64_t i = 0; i < dim; ++i) (dst_)[i] = 0;                                           \
                for (int o = 0; o < nobs; ++o) {                                                           \
                    const double w = row_weights ? row_weights[(int64_t)r * nobs + o] : 1.0;               \
                    for (int k = term_offsets[o]; k < term_offsets[o + 1]; ++k) {                          \
                        memcpy(tmp, (src_), (size_t)dim * sizeof(cplx));                                   \
                        apply_pauli(n, tmp, xmask[k], zmask[k]);                                           \
                        for (int64_t i = 0; i < dim; ++i) (dst_)[i] += w * coeff[k] * tmp[i];              \
                    }                                                                                      \
                }                                                                                          \
            } while (0)
        RUN_DIFF(psi, -1, -1);
        APPLY_O(Opsi, psi);
        for (int a = 0; a < nocc; ++a) {
            RUN_DIFF(pa + (int64_t)a * dim, a, -1);
            APPLY_O(Opa + (int64_t)a * dim, pa + (int64_t)a * dim);
        }
        cplx *pab = (cplx *)malloc((size_t)dim * sizeof(cplx));
        for (int a = 0; a < nocc; ++a)
            for (int b = a; b < nocc; ++b) {
                RUN_DIFF(pab, a, b);
                const double h = 2.0 * creal(inner(dim, pab, Opsi) + inner(dim, pa + (int64_t)a * dim,
                                                                        Opa + (int64_t)b * dim));
                const int p = pidx[og[a]] + ok[a], q = pidx[og[b]] + ok[b];
                acc[(int64_t)p * nparams + q] += h;
                if (a != b) acc[(int64_t)q * nparams + p] += h;
            }
        #undef RUN_DIFF
        #undef APPLY_O
        free(pab);
        free(psi);
        free(Opsi);
        free(tmp);
        free(pa);
        free(Opa);
    }
    memcpy(hess, acc, sizeof(double) * (size_t)nparams * nparams);
    free(acc);
    free(og);
    free(ok);
}

/* ------------------------------------------------------------------------ */
/* Density matrices and noise channels.                                      */
/* ------------------------------------------------------------------------ */

/* Kraus operators {K_k} (sum_k K_k^dagger K_k = I) of the single-qubit
 * channels, with probability p:
 *   bit flip:      sqrt(1-p) I, sqrt(p) X
 *   phase flip:    sqrt(1-p) I, sqrt(p) Z
 *   depolarizing:  sqrt(1-p) I, sqrt(p/3) X, sqrt(p/3) Y, sqrt(p/3) Z
 *   amplitude damping: [[1, 0], [0, sqrt(1-p)]], [[0, sqrt(p)], [0, 0]]
 * Returns the number of operators. */
static int kraus_ops(int kind, double p, cplx K[4][4])
{
    cplx I2[4] = {1, 0, 0, 1}, X[4] = {0, 1, 1, 0}, Y[4] = {0, -I, I, 0}, Z[4] = {1, 0, 0, -1};
    const double a = sqrt(1.0 - p);
    int nk = 0;
    switch (kind) {
    case O_BITFLIP:
        for (int e = 0; e < 4; ++e) { K[0][e] = a * I2[e]; K[1][e] = sqrt(p) * X[e]; }
        nk = 2;
        break;
    case O_PHASEFLIP:
        for (int e = 0; e < 4; ++e) { K[0][e] = a * I2[e]; K[1][e] = sqrt(p) * Z[e]; }
        nk = 2;
        break;
    case O_DEPOLARIZING: {
        const double b = sqrt(p / 3.0);
        for (int e = 0; e < 4; ++e) {
            K[0][e] = a * I2[e]; K[1][e] = b * X[e]; K[2][e] = b * Y[e]; K[3][e] = b * Z[e];
        }
        nk = 4;
        break;
    }
    default: /* amplitude damping */
        K[0][0] = 1; K[0][1] = 0; K[0][2] = 0; K[0][3] = a;
        K[1][0] = 0; K[1][1] = sqrt(p); K[1][2] = 0; K[1][3] = 0;
        nk = 2;
        break;
    }
    return nk;
}

static int is_noise(int kind)
{
    return kind == O_BITFLIP || kind == O_PHASEFLIP || kind == O_DEPOLARIZING || kind == O_AMPDAMP;
}

/* Operator applied from the left to every column of the dim x dim row-major
 * matrix m: op(v) acts on a column vector in place. */
typedef struct { int kind, w0, w1, w2; const double *t3; const cplx *blk; int dagger; } OracleOp;

static void op_apply(int n, cplx *v, const OracleOp *op)
{
    if (op->blk) apply_block(n, v, op->w0, -1, op->blk);
    else apply_gate(n, v, op->kind, op->w0, op->w1, op->w2, op->t3, op->dagger);
}

/* m <- A m A^dagger: A on every column, then conj(A) on every row (the rows
 * of m A^dagger are conj(A) applied to the rows of m; conj(A) v is formed as
 * conj(A conj(v))). */
static void sandwich(int n, cplx *m, const OracleOp *op, cplx *col)
{
    const int64_t dim = (int64_t)1 << n;
    for (int64_t j = 0; j < dim; ++j) {
        for (int64_t i = 0; i < dim; ++i) col[i] = m[i * dim + j];
        op_apply(n, col, op);
        for (int64_t i = 0; i < dim; ++i) m[i * dim + j] = col[i];
    }
    for (int64_t i = 0; i < dim; ++i) {
        cplx *row = m + i * dim;
        for (int64_t j = 0; j < dim; ++j) col[j] = conj(row[j]);
        op_apply(n, col, op);
        for (int64_t j = 0; j < dim; ++j) row[j] = conj(col[j]);
    }
}

/*
 * Mixed-state evolution rho_n = U_n ... U_1 rho_0 U_1^dagger ... U_n^dagger
 * (Sec. "Quantum Computing with Qubits", Background) from rho_0 = |0><0|,
 * with noise channels applied as rho -> sum_k K_k rho K_k^dagger, for every
 * batch row; then expect_out[row * nobs + o] = sum_k c_k Re Tr(P_k rho)
 * (Tr(P rho) = sum_i (P rho)_ii with P applied to every column).  rho_out
 * (batch x 2^n x 2^n, row-major, may be NULL) receives the matrices.
 */
void oracle_density(int n, int ngates, const int *kind, const int *w0, const int *w1, const int *w2,
                    const int *pidx, const int *didx, const double *angle,
                    const double *params, int nparams, const double *data, int nfeat, int batch,
                    const double *coeff, const uint64_t *xmask, const uint64_t *zmask,
                    const int *term_offsets, int nobs, double *expect_out, double *rho_out)
{
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) if (batch > 1)
    for (int r = 0; r < batch; ++r) {
        cplx *rho = (cplx *)calloc((size_t)(dim * dim), sizeof(cplx));
        cplx *acc = (cplx *)malloc((size_t)(dim * dim) * sizeof(cplx));
        cplx *tmp = (cplx *)malloc((size_t)(dim * dim) * sizeof(cplx));
        cplx *col = (cplx *)malloc((size_t)dim * sizeof(cplx));
        rho[0] = 1;
        for (int g = 0; g < ngates; ++g) {
            if (is_noise(kind[g])) {
                cplx K[4][4];
                const int nk = kraus_ops(kind[g], angle[g], K);
                for (int64_t i = 0; i < dim * dim; ++i) acc[i] = 0;
                for (int k = 0; k < nk; ++k) {
                    memcpy(tmp, rho, (size_t)(dim * dim) * sizeof(cplx));
                    OracleOp op = {0, w0[g], -1, -1, NULL, K[k], 0};
                    sandwich(n, tmp, &op, col);
                    for (int64_t i = 0; i < dim * dim; ++i) acc[i] += tmp[i];
                }
                memcpy(rho, acc, (size_t)(dim * dim) * sizeof(cplx));
            } else {
                double t3[3];
                gate_angles(g, kind[g], pidx, didx, angle, params, nparams, 0, data, nfeat, r, t3);
                OracleOp op = {kind[g], w0[g], w1[g], w2[g], t3, NULL, 0};
                sandwich(n, rho, &op, col);
            }
        }
        if (expect_out) {
            for (int o = 0; o < nobs; ++o) {
                double e = 0.0;
                for (int k = term_offsets[o]; k < term_offsets[o + 1]; ++k) {
                    double tr = 0.0;
                    for (int64_t j = 0; j < dim; ++j) {
                        for (int64_t i = 0; i < dim; ++i) col[i] = rho[i * dim + j];
                        apply_pauli(n, col, xmask[k], zmask[k]);
                        tr += creal(col[j]);
                    }
                    e += coeff[k] * tr;
                }
                expect_out[(int64_t)r * nobs + o] = e;
            }
        }
        if (rho_out) memcpy(rho_out + (int64_t)r * dim * dim * 2, rho, (size_t)(dim * dim) * sizeof(cplx));
        free(rho);
        free(acc);
        free(tmp);
        free(col);
    }
}

/* ------------------------------------------------------------------------ */
/* Shot sampling.                                                            */
/* ------------------------------------------------------------------------ */

/*
 * Outcomes of `shots` measurements of every row in the computational basis
 * (API Overview: measure(shots, wires)), by inversion of the cumulative
 * distribution (Devroye, "Non-Uniform Random Variate Generation", 1986,
 * Sec. III.2, the search done by bisection): with p_i = |psi_i|^2, C(i) = p_0 + ... +
 * p_i in index order and Z = C(2^n - 1), shot s returns the smallest i with
 * u_s * Z < C(i); when rounding leaves no such i it returns the last i with
 * p_i > 0.  wire_mask != 0 packs the bits of the selected wires of that
 * index, the lowest selected wire first (most significant).
 */
void oracle_sample(int n, int batch, const double *states_ri, int64_t shots, const double *uniforms,
                   uint64_t wire_mask, int64_t *out)
{
    const int64_t dim = (int64_t)1 << n;
    const cplx *states = (const cplx *)states_ri;
#pragma omp parallel for schedule(dynamic, 1) if (batch > 1)
    for (int r = 0; r < batch; ++r) {
        const cplx *psi = states + (int64_t)r * dim;
        double *cum = (double *)malloc((size_t)dim * sizeof(double));
        double run = 0.0;
        int64_t last_nz = dim - 1;
        for (int64_t i = 0; i < dim; ++i) {
            const double p = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
            run += p;
            cum[i] = run;
            if (p > 0.0) last_nz = i;
        }
        for (int64_t s = 0; s < shots; ++s) {
            const double target = uniforms[(int64_t)r * shots + s] * cum[dim - 1];
            /* smallest i with target < C(i): bisection on the non-decreasing C */
            int64_t lo = 0, hi = dim;
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (target < cum[mid]) hi = mid;
                else lo = mid + 1;
            }
            const int64_t idx = lo < dim ? lo : last_nz;
            int64_t o = idx;
            if (wire_mask) {
                o = 0;
                for (int q = 0; q < n; ++q)
                    if ((wire_mask >> q) & 1) o = (o << 1) | ((idx >> bitpos(n, q)) & 1);
            }
            out[(int64_t)r * shots + s] = o;
        }
        free(cum);
    }
}

/* ------------------------------------------------------------------------ */
/* Dense matrix on the lowest-order wires.                                   */
/* ------------------------------------------------------------------------ */

/* psi <- (I (x) U) psi for every row, U a 2^nw x 2^nw matrix (row-major,
 * interleaved re/im) on the nw lowest-order wires n-nw .. n-1.  With wire 0 as
 * the most significant index bit, those wires are the low nw bits, so each
 * row splits into 2^(n-nw) contiguous groups of 2^nw amplitudes and U
 * multiplies each group as a vector: y_i = sum_j U_ij x_j. */
void oracle_apply_dense(int n, int nw, const double *u, int batch, double *states)
{
    const int64_t bw = (int64_t)1 << nw;
    const int64_t groups = (int64_t)batch << (n - nw);
    const cplx *U = (const cplx *)u;
    cplx *st = (cplx *)states;
#pragma omp parallel
    {
        cplx *y = (cplx *)malloc((size_t)bw * sizeof(cplx));
#pragma omp for schedule(static)
        for (int64_t v = 0; v < groups; ++v) {
            cplx *x = st + v * bw;
            for (int64_t i = 0; i < bw; ++i) {
                cplx acc = 0;
                for (int64_t j = 0; j < bw; ++j) acc += U[i * bw + j] * x[j];
                y[i] = acc;
            }
            memcpy(x, y, (size_t)bw * sizeof(cplx));
        }
        free(y);
    }
}
