/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the global stiffness-matrix build.
 *
 * TEST INFRASTRUCTURE, NOT THE PRODUCT.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark load this file's library.  It shares no
 * code, header, table or constant with the CUDA library and includes none of it.
 *
 * What it computes (Ramirez-Gil, Tsuzuki, Montealegre-Rubio, "Global finite
 * element matrix construction based on a CPU-GPU implementation"):
 *   - the element matrix of the Poisson operator div(c grad phi) = 0
 *     (Eq. 2), k_e = c * integral B^T B dOmega (Eq. 7), mapped to the
 *     reference cube (Eq. 8) and evaluated by 2x2x2 Gauss-Legendre quadrature
 *     (Eq. 9) for the 8-node trilinear brick, one point per loop level in the
 *     order r (outer), s, t (inner);
 *   - the same for the 4-node linear tetrahedron with the exact 1-point rule
 *     (k_e = c |det J| / 6 * B^T B);
 *   - Algorithm 1: a loop over elements that writes, for each element, the
 *     triplets (row, col, val) of its lower triangle (Section 3: only the 36
 *     entries a >= b of the symmetric 8x8 matrix are kept), followed by one
 *     sparse conversion (Section 3, assembly as a format conversion): a stable
 *     sort by (row, col) and a sum of repeated entries in emission order
 *     (footnote on the triplet format), giving a lower-triangular CSR matrix.
 *   - Eq. 6 as the sum K = sum_e k_e is exactly what that conversion produces.
 *   - the mass matrix m_e = c * integral N^T N (the generalisation of Section 5)
 *     and the load vector of a per-element source (Section 1, steps (ii)-(iii));
 *   - linear isotropic elasticity, three DOFs per node (Algorithm 1's DOFxn),
 *     k_e = integral Be^T D Be with the same quadrature, assembled through the
 *     same triplets and conversion over DOFs;
 *   - the gradient of L = sum over stored entries of G_ij K_ij with respect to
 *     the node coordinates, by the complex-step derivative of the element
 *     routine, and with respect to c_e (k_e is linear in c_e).
 *
 * Readings of points the paper leaves open (each is stated where it is used):
 *   node order of the brick, the packed order of the lower triangle, the use of
 *   |det J|, storage of a local pair (a, b) at (max(g_a, g_b), min(g_a, g_b)).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Natural coordinates of the brick's nodes: nodes 0-3 on t = -1
 * counter-clockwise from (-1,-1,-1), nodes 4-7 the same on t = +1. */
static const double BRICK_NODES[8][3] = {
    {-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
    {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

/* Reference gradients of the tetrahedron's barycentric functions:
 * lambda_0 = 1 - xi - eta - zeta, lambda_i = xi_i.  TET_DL[i][a] = d lambda_a / d xi_i. */
static const double TET_DL[3][4] = {{-1, 1, 0, 0}, {-1, 0, 1, 0}, {-1, 0, 0, 1}};

/*
 * Element routines, written once and instantiated for double and for
 * double complex (the latter only for the complex-step derivative).  The body
 * is the plain definition: shape-function derivatives dN at the point, the
 * Jacobian J = dN * X_e (J_ij = d x_j / d xi_i, Section 3), det J by the 3x3
 * formula, J^{-1} = adj(J) / det J, B = J^{-1} dN, and k += c w |det J| B^T B.
 * The sign of det J is read from its real part so that the complex instance
 * stays analytic.  Returns the number of points with det J <= 0.
 */
#define DEFINE_ELEMENT_ROUTINES(SUFFIX, T, RE)                                              \
    static void inv3_##SUFFIX(const T J[3][3], T *det, T inv[3][3]) {                       \
        T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];                                      \
        T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];                                      \
        T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];                                      \
        T c10 = J[0][2] * J[2][1] - J[0][1] * J[2][2];                                      \
        T c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];                                      \
        T c12 = J[0][1] * J[2][0] - J[0][0] * J[2][1];                                      \
        T c20 = J[0][1] * J[1][2] - J[0][2] * J[1][1];                                      \
        T c21 = J[0][2] * J[1][0] - J[0][0] * J[1][2];                                      \
        T c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];                                      \
        T d = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;                                \
        *det = d;                                                                           \
        /* inverse = transpose of the cofactor matrix over det */                           \
        inv[0][0] = c00 / d; inv[0][1] = c10 / d; inv[0][2] = c20 / d;                      \
        inv[1][0] = c01 / d; inv[1][1] = c11 / d; inv[1][2] = c21 / d;                      \
        inv[2][0] = c02 / d; inv[2][1] = c12 / d; inv[2][2] = c22 / d;                      \
    }                                                                                       \
                                                                                            \
    static int ke_brick_##SUFFIX(const T xe[24], T c, T ke[64]) {                           \
        const double g = 1.0 / sqrt(3.0);                                                   \
        const double pts[2] = {-g, g};                                                      \
        int nonpos = 0;                                                                     \
        for (int i = 0; i < 64; ++i) ke[i] = 0;                                             \
        for (int ir = 0; ir < 2; ++ir)                                                      \
            for (int is = 0; is < 2; ++is)                                                  \
                for (int it = 0; it < 2; ++it) {                                            \
                    const double r = pts[ir], s = pts[is], t = pts[it];                     \
                    double dN[3][8];                                                        \
                    for (int a = 0; a < 8; ++a) {                                           \
                        const double ra = BRICK_NODES[a][0], sa = BRICK_NODES[a][1],        \
                                     ta = BRICK_NODES[a][2];                                \
                        /* N_a = (1 + r r_a)(1 + s s_a)(1 + t t_a) / 8 */                   \
                        dN[0][a] = 0.125 * ra * (1 + s * sa) * (1 + t * ta);                \
                        dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + t * ta);                \
                        dN[2][a] = 0.125 * ta * (1 + r * ra) * (1 + s * sa);                \
                    }                                                                       \
                    T J[3][3];                                                              \
                    for (int i = 0; i < 3; ++i)                                             \
                        for (int j = 0; j < 3; ++j) {                                       \
                            T acc = 0;                                                      \
                            for (int a = 0; a < 8; ++a) acc += dN[i][a] * xe[3 * a + j];    \
                            J[i][j] = acc;                                                  \
                        }                                                                   \
                    T det, inv[3][3];                                                       \
                    inv3_##SUFFIX(J, &det, inv);                                            \
                    if (RE(det) <= 0) ++nonpos;                                             \
                    T absdet = RE(det) < 0 ? -det : det; /* |J| of Eq. 8, weights 1 */      \
                    T B[3][8];                                                              \
                    for (int i = 0; i < 3; ++i)                                             \
                        for (int a = 0; a < 8; ++a) {                                       \
                            T acc = 0;                                                      \
                            for (int k = 0; k < 3; ++k) acc += inv[i][k] * dN[k][a];        \
                            B[i][a] = acc;                                                  \
                        }                                                                   \
                    for (int a = 0; a < 8; ++a)                                             \
                        for (int b = 0; b < 8; ++b) {                                       \
                            T acc = 0;                                                      \
                            for (int i = 0; i < 3; ++i) acc += B[i][a] * B[i][b];           \
                            ke[8 * a + b] += c * absdet * acc;                              \
                        }                                                                   \
                }                                                                           \
        return nonpos;                                                                      \
    }                                                                                       \
                                                                                            \
    static int ke_tet_##SUFFIX(const T xe[12], T c, T ke[16]) {                             \
        T J[3][3];                                                                          \
        for (int i = 0; i < 3; ++i)                                                         \
            for (int j = 0; j < 3; ++j) J[i][j] = xe[3 * (i + 1) + j] - xe[j];              \
        T det, inv[3][3];                                                                   \
        inv3_##SUFFIX(J, &det, inv);                                                        \
        T vol = (RE(det) < 0 ? -det : det) / 6.0;                                           \
        T B[3][4];                                                                          \
        for (int i = 0; i < 3; ++i)                                                         \
            for (int a = 0; a < 4; ++a) {                                                   \
                T acc = 0;                                                                  \
                for (int k = 0; k < 3; ++k) acc += inv[i][k] * TET_DL[k][a];                \
                B[i][a] = acc;                                                              \
            }                                                                               \
        for (int a = 0; a < 4; ++a)                                                         \
            for (int b = 0; b < 4; ++b) {                                                   \
                T acc = 0;                                                                  \
                for (int i = 0; i < 3; ++i) acc += B[i][a] * B[i][b];                       \
                ke[4 * a + b] = c * vol * acc;                                              \
            }                                                                               \
        return RE(det) <= 0 ? 1 : 0;                                                        \
    }

static double re_d(double x) { return x; }
static double re_z(double complex x) { return creal(x); }
DEFINE_ELEMENT_ROUTINES(d, double, re_d)
DEFINE_ELEMENT_ROUTINES(z, double complex, re_z)

/*
 * The mass matrix of the same elements, M_ab = integral c N_a N_b dOmega: the
 * other operator the paper says its construction generalises to (Section 5,
 * Conclusions).  The brick uses the same 2x2x2 Gauss rule and the same |det J|
 * of Eq. 8 as k_e; the tetrahedron the 4-point rule that is exact for
 * quadratics (barycentric points (a, b, b, b) and its permutations,
 * a = (5 + 3 sqrt 5) / 20, b = (5 - sqrt 5) / 20, each weighted by a quarter of
 * the volume).  Returns the number of points with det J <= 0.
 */
static int me_brick(const double xe[24], double c, double me[64]) {
    const double g = 1.0 / sqrt(3.0);
    const double pts[2] = {-g, g};
    int nonpos = 0;
    for (int i = 0; i < 64; ++i) me[i] = 0;
    for (int ir = 0; ir < 2; ++ir)
        for (int is = 0; is < 2; ++is)
            for (int it = 0; it < 2; ++it) {
                const double r = pts[ir], s = pts[is], t = pts[it];
                double N[8], dN[3][8];
                for (int a = 0; a < 8; ++a) {
                    const double ra = BRICK_NODES[a][0], sa = BRICK_NODES[a][1], ta = BRICK_NODES[a][2];
                    N[a] = 0.125 * (1 + r * ra) * (1 + s * sa) * (1 + t * ta);
                    dN[0][a] = 0.125 * ra * (1 + s * sa) * (1 + t * ta);
                    dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + t * ta);
                    dN[2][a] = 0.125 * ta * (1 + r * ra) * (1 + s * sa);
                }
                double J[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double acc = 0;
                        for (int a = 0; a < 8; ++a) acc += dN[i][a] * xe[3 * a + j];
                        J[i][j] = acc;
                    }
                double det, inv[3][3];
                inv3_d(J, &det, inv);
                if (det <= 0) ++nonpos;
                const double absdet = fabs(det);
                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b < 8; ++b) me[8 * a + b] += c * absdet * N[a] * N[b];
            }
    return nonpos;
}

static int me_tet(const double xe[12], double c, double me[16]) {
    double J[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] = xe[3 * (i + 1) + j] - xe[j];
    double det, inv[3][3];
    inv3_d(J, &det, inv);
    const double vol = fabs(det) / 6.0;
    const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0, qb = (5.0 - sqrt(5.0)) / 20.0;
    for (int i = 0; i < 16; ++i) me[i] = 0;
    for (int q = 0; q < 4; ++q) {
        double lam[4];
        for (int a = 0; a < 4; ++a) lam[a] = a == q ? qa : qb;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) me[4 * a + b] += c * (vol / 4.0) * lam[a] * lam[b];
    }
    return det <= 0 ? 1 : 0;
}

/*
 * Linear isotropic elasticity: the vector problem with three degrees of freedom
 * per node (Algorithm 1 maps local to global DOFs through the number of DOFs per
 * node, DOFxn; the paper itself only builds the scalar case, Section 3).  The
 * operator is the textbook one, not taken from the paper:
 *   k_e = integral Be^T D Be dOmega,
 * Be the 6 x 3npe strain-displacement matrix in Voigt order (e_xx, e_yy, e_zz,
 * g_xy, g_yz, g_zx, engineering shears g = 2 e) built from the physical
 * gradients B = J^{-1} dN of the scalar routine, and D the isotropic material
 * matrix of the element's Lame parameters (lambda, mu): lambda + 2 mu on the
 * normal diagonal, lambda off it, mu on the shear diagonal.  Local DOF 3a + i is
 * component i of node a.  Same Gauss rule, |det J| and node order as k_e of
 * Eq. 9; the tetrahedron's integrand is constant (1 point, weight 1/6).
 * ke is the dense (3npe) x (3npe) matrix.  Returns the number of points with
 * det J <= 0.
 */
static void elastic_add(int npe, const double B[3][8], double w, double lam, double mu, double *ke) {
    const int nk = 3 * npe;
    double Be[6][24];
    for (int k = 0; k < 6; ++k)
        for (int A = 0; A < nk; ++A) Be[k][A] = 0.0;
    for (int a = 0; a < npe; ++a) {
        Be[0][3 * a + 0] = B[0][a];
        Be[1][3 * a + 1] = B[1][a];
        Be[2][3 * a + 2] = B[2][a];
        Be[3][3 * a + 0] = B[1][a]; Be[3][3 * a + 1] = B[0][a];
        Be[4][3 * a + 1] = B[2][a]; Be[4][3 * a + 2] = B[1][a];
        Be[5][3 * a + 0] = B[2][a]; Be[5][3 * a + 2] = B[0][a];
    }
    double D[6][6];
    for (int k = 0; k < 6; ++k)
        for (int l = 0; l < 6; ++l) D[k][l] = 0.0;
    for (int k = 0; k < 3; ++k) {
        for (int l = 0; l < 3; ++l) D[k][l] = lam;
        D[k][k] = lam + 2.0 * mu;
        D[k + 3][k + 3] = mu;
    }
    for (int A = 0; A < nk; ++A)
        for (int Bc = 0; Bc < nk; ++Bc) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k)
                for (int l = 0; l < 6; ++l) acc += Be[k][A] * D[k][l] * Be[l][Bc];
            ke[nk * A + Bc] += w * acc;
        }
}

static int ke_elastic(int npe, const double *xe, double lam, double mu, double *ke) {
    const int nk = 3 * npe;
    int nonpos = 0;
    for (int i = 0; i < nk * nk; ++i) ke[i] = 0.0;
    if (npe == 8) {
        const double g = 1.0 / sqrt(3.0);
        const double pts[2] = {-g, g};
        for (int ir = 0; ir < 2; ++ir)
            for (int is = 0; is < 2; ++is)
                for (int it = 0; it < 2; ++it) {
                    const double r = pts[ir], s = pts[is], t = pts[it];
                    double dN[3][8];
                    for (int a = 0; a < 8; ++a) {
                        const double ra = BRICK_NODES[a][0], sa = BRICK_NODES[a][1], ta = BRICK_NODES[a][2];
                        dN[0][a] = 0.125 * ra * (1 + s * sa) * (1 + t * ta);
                        dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + t * ta);
                        dN[2][a] = 0.125 * ta * (1 + r * ra) * (1 + s * sa);
                    }
                    double J[3][3];
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            double acc = 0;
                            for (int a = 0; a < 8; ++a) acc += dN[i][a] * xe[3 * a + j];
                            J[i][j] = acc;
                        }
                    double det, inv[3][3], B[3][8];
                    inv3_d(J, &det, inv);
                    if (det <= 0) ++nonpos;
                    for (int i = 0; i < 3; ++i)
                        for (int a = 0; a < 8; ++a) {
                            double acc = 0;
                            for (int k = 0; k < 3; ++k) acc += inv[i][k] * dN[k][a];
                            B[i][a] = acc;
                        }
                    elastic_add(8, B, fabs(det), lam, mu, ke);
                }
    } else {
        double J[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) J[i][j] = xe[3 * (i + 1) + j] - xe[j];
        double det, inv[3][3], B[3][8];
        inv3_d(J, &det, inv);
        if (det <= 0) ++nonpos;
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 4; ++a) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += inv[i][k] * TET_DL[k][a];
                B[i][a] = acc;
            }
        elastic_add(4, B, fabs(det) / 6.0, lam, mu, ke);
    }
    return nonpos;
}

/* The same elasticity element in complex arithmetic (for the complex-step
 * derivative of the backward pass); the sign of det J from its real part. */
static void elastic_add_z(int npe, const double complex B[3][8], double complex w, double lam, double mu,
                          double complex *ke) {
    const int nk = 3 * npe;
    double complex Be[6][24];
    for (int k = 0; k < 6; ++k)
        for (int A = 0; A < nk; ++A) Be[k][A] = 0.0;
    for (int a = 0; a < npe; ++a) {
        Be[0][3 * a + 0] = B[0][a];
        Be[1][3 * a + 1] = B[1][a];
        Be[2][3 * a + 2] = B[2][a];
        Be[3][3 * a + 0] = B[1][a]; Be[3][3 * a + 1] = B[0][a];
        Be[4][3 * a + 1] = B[2][a]; Be[4][3 * a + 2] = B[1][a];
        Be[5][3 * a + 0] = B[2][a]; Be[5][3 * a + 2] = B[0][a];
    }
    double D[6][6];
    for (int k = 0; k < 6; ++k)
        for (int l = 0; l < 6; ++l) D[k][l] = 0.0;
    for (int k = 0; k < 3; ++k) {
        for (int l = 0; l < 3; ++l) D[k][l] = lam;
        D[k][k] = lam + 2.0 * mu;
        D[k + 3][k + 3] = mu;
    }
    for (int A = 0; A < nk; ++A)
        for (int Bc = 0; Bc < nk; ++Bc) {
            double complex acc = 0.0;
            for (int k = 0; k < 6; ++k)
                for (int l = 0; l < 6; ++l) acc += Be[k][A] * D[k][l] * Be[l][Bc];
            ke[nk * A + Bc] += w * acc;
        }
}

static void ke_elastic_z(int npe, const double complex *xe, double lam, double mu, double complex *ke) {
    const int nk = 3 * npe;
    for (int i = 0; i < nk * nk; ++i) ke[i] = 0.0;
    if (npe == 8) {
        const double g = 1.0 / sqrt(3.0);
        const double pts[2] = {-g, g};
        for (int ir = 0; ir < 2; ++ir)
            for (int is = 0; is < 2; ++is)
                for (int it = 0; it < 2; ++it) {
                    const double r = pts[ir], s = pts[is], t = pts[it];
                    double dN[3][8];
                    for (int a = 0; a < 8; ++a) {
                        const double ra = BRICK_NODES[a][0], sa = BRICK_NODES[a][1], ta = BRICK_NODES[a][2];
                        dN[0][a] = 0.125 * ra * (1 + s * sa) * (1 + t * ta);
                        dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + t * ta);
                        dN[2][a] = 0.125 * ta * (1 + r * ra) * (1 + s * sa);
                    }
                    double complex J[3][3];
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            double complex acc = 0;
                            for (int a = 0; a < 8; ++a) acc += dN[i][a] * xe[3 * a + j];
                            J[i][j] = acc;
                        }
                    double complex det, inv[3][3], B[3][8];
                    inv3_z(J, &det, inv);
                    for (int i = 0; i < 3; ++i)
                        for (int a = 0; a < 8; ++a) {
                            double complex acc = 0;
                            for (int k = 0; k < 3; ++k) acc += inv[i][k] * dN[k][a];
                            B[i][a] = acc;
                        }
                    elastic_add_z(8, B, creal(det) < 0 ? -det : det, lam, mu, ke);
                }
    } else {
        double complex J[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) J[i][j] = xe[3 * (i + 1) + j] - xe[j];
        double complex det, inv[3][3], B[3][8];
        inv3_z(J, &det, inv);
        for (int i = 0; i < 3; ++i)
            for (int a = 0; a < 4; ++a) {
                double complex acc = 0;
                for (int k = 0; k < 3; ++k) acc += inv[i][k] * TET_DL[k][a];
                B[i][a] = acc;
            }
        elastic_add_z(4, B, (creal(det) < 0 ? -det : det) / 6.0, lam, mu, ke);
    }
}

/* Operators: 0 = stiffness k_e (Eq. 9), 1 = mass m_e, 2 = elasticity (3 DOFs per
 * node).  cv = the element's coefficients: c_e, or (lambda_e, mu_e) for op 2. */
static int op_dofs(int op) { return op == 2 ? 3 : 1; }

static int element_dense(int op, int npe, const double *xe, const double *cv, double *ke) {
    if (op == 2) return ke_elastic(npe, xe, cv[0], cv[1], ke);
    if (op == 1) return npe == 8 ? me_brick(xe, cv[0], ke) : me_tet(xe, cv[0], ke);
    return npe == 8 ? ke_brick_d(xe, cv[0], ke) : ke_tet_d(xe, cv[0], ke);
}

/* Full dense element matrix of one element (row-major npe x npe), ops 0 and 1. */
int oracle_ke_dense(int op, int npe, const double *xe, double c, double *ke) {
    if ((npe != 8 && npe != 4) || (op != 0 && op != 1)) return -1;
    return element_dense(op, npe, xe, &c, ke);
}

/* Dense (3npe) x (3npe) elasticity matrix of one element (op 2). */
int oracle_ke_elastic_dense(int npe, const double *xe, double lam, double mu, double *ke) {
    if (npe != 8 && npe != 4) return -1;
    return ke_elastic(npe, xe, lam, mu, ke);
}

static void gather(int npe, const int32_t *E, const double *X, int64_t e, double *xe) {
    for (int a = 0; a < npe; ++a) {
        const int64_t g = E[e * npe + a];
        xe[3 * a + 0] = X[3 * g + 0];
        xe[3 * a + 1] = X[3 * g + 1];
        xe[3 * a + 2] = X[3 * g + 2];
    }
}

/*
 * Packed lower triangle of every element matrix of operator op: with nk = DOFs
 * per element (npe, or 3 npe for op 2), entry p = A(A+1)/2 + B for B <= A
 * (row-major lower order over local DOFs).  c holds one coefficient per element,
 * two (lambda, mu) for op 2.  cs[p] = sqrt(k_AA k_BB), the Cauchy-Schwarz bound
 * of |k_AB| for the positive semidefinite k_e (or m_e), used to scale errors.
 * Returns the number of elements with some det J <= 0.
 */
int64_t oracle_ke_packed(int op, int npe, int64_t n_elems, const int32_t *E, const double *X,
                         const double *c, double *ke_out, double *cs_out) {
    const int nk = op_dofs(op) * npe, np = nk * (nk + 1) / 2, nc = op == 2 ? 2 : 1;
    int64_t bad = 0;
    double xe[24], ke[576];
    for (int64_t e = 0; e < n_elems; ++e) {
        gather(npe, E, X, e, xe);
        if (element_dense(op, npe, xe, c + nc * e, ke) > 0) ++bad;
        for (int a = 0; a < nk; ++a)
            for (int b = 0; b <= a; ++b) {
                const int p = a * (a + 1) / 2 + b;
                ke_out[e * np + p] = ke[nk * a + b];
                if (cs_out) cs_out[e * np + p] = sqrt(fabs(ke[nk * a + a] * ke[nk * b + b]));
            }
    }
    return bad;
}

/*
 * Algorithm 1, the element loop: for every element (in element order) compute k_e and
 * write its triplets.  Mapping(E(e), DOFxn): local DOF A = DOFxn a + i of node a
 * is global DOF DOFxn g_a + i (components of a node adjacent).  The local pair
 * (A, B), B <= A, goes to global (max(G_A, G_B), min(G_A, G_B)) with value
 * k_e[A][B] (k_e is symmetric).  rows/cols/vals/cs have room for
 * n_elems * nk(nk+1)/2 entries.
 */
int64_t oracle_triplets(int op, int npe, int64_t n_elems, const int32_t *E, const double *X,
                        const double *c, int64_t *rows, int32_t *cols, double *vals, double *cs) {
    const int dofxn = op_dofs(op), nk = dofxn * npe, np = nk * (nk + 1) / 2, nc = op == 2 ? 2 : 1;
    int64_t bad = 0;
    double xe[24], ke[576];
    for (int64_t e = 0; e < n_elems; ++e) {
        gather(npe, E, X, e, xe);
        if (element_dense(op, npe, xe, c + nc * e, ke) > 0) ++bad;
        for (int a = 0; a < nk; ++a)
            for (int b = 0; b <= a; ++b) {
                const int64_t t = e * np + a * (a + 1) / 2 + b;
                const int32_t ga = dofxn * E[e * npe + a / dofxn] + a % dofxn;
                const int32_t gb = dofxn * E[e * npe + b / dofxn] + b % dofxn;
                rows[t] = ga > gb ? ga : gb;
                cols[t] = ga > gb ? gb : ga;
                vals[t] = ke[nk * a + b];
                cs[t] = sqrt(fabs(ke[nk * a + a] * ke[nk * b + b]));
            }
    }
    return bad;
}

/* Stable merge sort of idx[] by key[idx] (bottom-up, ties keep input order). */
static void stable_sort_by_key(int64_t n, const int64_t *key, int64_t *idx) {
    int64_t *tmp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *src = idx, *dst = tmp;
    for (int64_t width = 1; width < n; width *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * width) {
            int64_t mid = lo + width < n ? lo + width : n;
            int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int64_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi) dst[k++] = (key[src[j]] < key[src[i]]) ? src[j++] : src[i++];
            while (i < mid) dst[k++] = src[i++];
            while (j < hi) dst[k++] = src[j++];
        }
        int64_t *s = src; src = dst; dst = s;
    }
    if (src != idx) memcpy(idx, src, (size_t)n * sizeof(int64_t));
    free(tmp);
}

/*
 * Algorithm 1, the sparse conversion after the element loop.  Sort the triplets by
 * (row, col), stably, and sum repeated (row, col) entries in emission order.
 * Output lower-triangular CSR: rowptr[n_nodes + 1], col ascending within a row.
 * abs_out = sum of |val|, cs_out = sum of cs over the merged triplets;
 * slot[t] = CSR position of triplet t.  Returns nnz.
 */
int64_t oracle_compress(int64_t ntrip, int64_t n_nodes, const int64_t *rows, const int32_t *cols,
                        const double *vals, const double *cs, int64_t *rowptr, int32_t *col_out,
                        double *val_out, double *abs_out, double *cs_out, int64_t *slot) {
    int64_t *key = (int64_t *)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int64_t));
    int64_t *idx = (int64_t *)malloc((size_t)(ntrip > 0 ? ntrip : 1) * sizeof(int64_t));
    for (int64_t t = 0; t < ntrip; ++t) {
        key[t] = rows[t] * n_nodes + cols[t];
        idx[t] = t;
    }
    stable_sort_by_key(ntrip, key, idx);
    for (int64_t i = 0; i <= n_nodes; ++i) rowptr[i] = 0;
    int64_t nnz = 0;
    for (int64_t u = 0; u < ntrip; ++u) {
        const int64_t t = idx[u];
        if (u == 0 || key[t] != key[idx[u - 1]]) {
            col_out[nnz] = cols[t];
            val_out[nnz] = 0.0;
            abs_out[nnz] = 0.0;
            cs_out[nnz] = 0.0;
            rowptr[rows[t] + 1] += 1;
            ++nnz;
        }
        val_out[nnz - 1] += vals[t];
        abs_out[nnz - 1] += fabs(vals[t]);
        cs_out[nnz - 1] += cs[t];
        if (slot) slot[t] = nnz - 1;
    }
    for (int64_t i = 0; i < n_nodes; ++i) rowptr[i + 1] += rowptr[i];
    free(key);
    free(idx);
    return nnz;
}

/*
 * Global load vector of a per-element constant source s_e (Section 1, steps (ii)
 * and (iii): the local load vectors f_e and their assembly into F, the step the
 * paper sets aside):
 *   f_e,a = src_e * integral over the element of N_a,
 * the brick by the same 2x2x2 Gauss rule and |det J| as k_e, the tetrahedron by the
 * 4-point rule of the mass matrix; F[E[e][a]] += f_e,a in element order.  F must be
 * zeroed by the caller.  Returns the number of elements with some det J <= 0.
 */
int64_t oracle_load(int npe, int64_t n_elems, const int32_t *E, const double *X, const double *src, double *F) {
    int64_t bad = 0;
    double xe[24];
    for (int64_t e = 0; e < n_elems; ++e) {
        gather(npe, E, X, e, xe);
        double fe[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int nonpos = 0;
        if (npe == 8) {
            const double g = 1.0 / sqrt(3.0);
            const double pts[2] = {-g, g};
            for (int ir = 0; ir < 2; ++ir)
                for (int is = 0; is < 2; ++is)
                    for (int it = 0; it < 2; ++it) {
                        const double r = pts[ir], s = pts[is], t = pts[it];
                        double N[8], dN[3][8];
                        for (int a = 0; a < 8; ++a) {
                            const double ra = BRICK_NODES[a][0], sa = BRICK_NODES[a][1], ta = BRICK_NODES[a][2];
                            N[a] = 0.125 * (1 + r * ra) * (1 + s * sa) * (1 + t * ta);
                            dN[0][a] = 0.125 * ra * (1 + s * sa) * (1 + t * ta);
                            dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + t * ta);
                            dN[2][a] = 0.125 * ta * (1 + r * ra) * (1 + s * sa);
                        }
                        double J[3][3];
                        for (int i = 0; i < 3; ++i)
                            for (int j = 0; j < 3; ++j) {
                                double acc = 0;
                                for (int a = 0; a < 8; ++a) acc += dN[i][a] * xe[3 * a + j];
                                J[i][j] = acc;
                            }
                        double det, inv[3][3];
                        inv3_d(J, &det, inv);
                        if (det <= 0) nonpos = 1;
                        for (int a = 0; a < 8; ++a) fe[a] += src[e] * fabs(det) * N[a];
                    }
        } else {
            double J[3][3];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) J[i][j] = xe[3 * (i + 1) + j] - xe[j];
            double det, inv[3][3];
            inv3_d(J, &det, inv);
            if (det <= 0) nonpos = 1;
            const double vol = fabs(det) / 6.0;
            const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0, qb = (5.0 - sqrt(5.0)) / 20.0;
            for (int q = 0; q < 4; ++q)
                for (int a = 0; a < 4; ++a) fe[a] += src[e] * (vol / 4.0) * (a == q ? qa : qb);
        }
        bad += nonpos;
        for (int a = 0; a < npe; ++a) F[E[e * npe + a]] += fe[a];
    }
    return bad;
}

/*
 * The mass matrix of the brick and the tetrahedron in complex arithmetic, the
 * same steps as me_brick and me_tet, for the complex-step derivative below.  The
 * sign of det J is read from its real part.
 */
static void me_brick_z(const double complex xe[24], double complex c, double complex me[64]) {
    const double g = 1.0 / sqrt(3.0);
    const double pts[2] = {-g, g};
    for (int i = 0; i < 64; ++i) me[i] = 0;
    for (int ir = 0; ir < 2; ++ir)
        for (int is = 0; is < 2; ++is)
            for (int it = 0; it < 2; ++it) {
                const double r = pts[ir], s = pts[is], t = pts[it];
                double N[8], dN[3][8];
                for (int a = 0; a < 8; ++a) {
                    const double ra = BRICK_NODES[a][0], sa = BRICK_NODES[a][1], ta = BRICK_NODES[a][2];
                    N[a] = 0.125 * (1 + r * ra) * (1 + s * sa) * (1 + t * ta);
                    dN[0][a] = 0.125 * ra * (1 + s * sa) * (1 + t * ta);
                    dN[1][a] = 0.125 * sa * (1 + r * ra) * (1 + t * ta);
                    dN[2][a] = 0.125 * ta * (1 + r * ra) * (1 + s * sa);
                }
                double complex J[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double complex acc = 0;
                        for (int a = 0; a < 8; ++a) acc += dN[i][a] * xe[3 * a + j];
                        J[i][j] = acc;
                    }
                double complex det, inv[3][3];
                inv3_z(J, &det, inv);
                const double complex absdet = creal(det) < 0 ? -det : det;
                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b < 8; ++b) me[8 * a + b] += c * absdet * N[a] * N[b];
            }
}

static void me_tet_z(const double complex xe[12], double complex c, double complex me[16]) {
    double complex J[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] = xe[3 * (i + 1) + j] - xe[j];
    double complex det, inv[3][3];
    inv3_z(J, &det, inv);
    const double complex vol = (creal(det) < 0 ? -det : det) / 6.0;
    const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0, qb = (5.0 - sqrt(5.0)) / 20.0;
    for (int i = 0; i < 16; ++i) me[i] = 0;
    for (int q = 0; q < 4; ++q) {
        double lam[4];
        for (int a = 0; a < 4; ++a) lam[a] = a == q ? qa : qb;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) me[4 * a + b] += c * (vol / 4.0) * lam[a] * lam[b];
    }
}

/*
 * Gradient of L = sum_(e, p) S[e, p] * k_e[p] over the packed lower entries p of
 * every element (S is the upstream value G_ij of the CSR entry that (e, p) lands
 * in), for operator op (0 stiffness, 1 mass).  dc[e] = sum_p S[e, p] k_e[p] / c_e
 * because k_e is linear in c_e.  dX[g] += d L / d x_g by the complex-step
 * derivative Im L(x + i h e_j) / h of the element routine (exact up to rounding
 * for this analytic function).  dX must be zeroed by the caller.
 */
static void elastic_vjp(int npe, int64_t n_elems, const int32_t *E, const double *X, const double *c,
                        const double *S, double *dX, double *dc);

void oracle_vjp_op(int op, int npe, int64_t n_elems, const int32_t *E, const double *X, const double *c,
                   const double *S, double *dX, double *dc) {
    if (op == 2) {
        elastic_vjp(npe, n_elems, E, X, c, S, dX, dc);
        return;
    }
    const int np = npe * (npe + 1) / 2;
    double xe[24], ke[64];
    double complex xz[24], kz[64];
    for (int64_t e = 0; e < n_elems; ++e) {
        gather(npe, E, X, e, xe);
        const double one = 1.0;
        element_dense(op, npe, xe, &one, ke);
        double l1 = 0.0;
        for (int a = 0; a < npe; ++a)
            for (int b = 0; b <= a; ++b) l1 += S[e * np + a * (a + 1) / 2 + b] * ke[npe * a + b];
        dc[e] = l1;
        for (int k = 0; k < 3 * npe; ++k) {
            const double h = 1e-30 * (fabs(xe[k]) > 1.0 ? fabs(xe[k]) : 1.0);
            for (int m = 0; m < 3 * npe; ++m) xz[m] = xe[m];
            xz[k] += h * I;
            if (op == 1) {
                if (npe == 8) me_brick_z(xz, c[e], kz); else me_tet_z(xz, c[e], kz);
            } else {
                if (npe == 8) ke_brick_z(xz, c[e], kz); else ke_tet_z(xz, c[e], kz);
            }
            double dl = 0.0;
            for (int a = 0; a < npe; ++a)
                for (int b = 0; b <= a; ++b)
                    dl += S[e * np + a * (a + 1) / 2 + b] * cimag(kz[npe * a + b]) / h;
            dX[3 * (int64_t)E[e * npe + k / 3] + k % 3] += dl;
        }
    }
}

/* The stiffness operator's gradient (op 0 of oracle_vjp_op). */
void oracle_vjp(int npe, int64_t n_elems, const int32_t *E, const double *X, const double *c,
                const double *S, double *dX, double *dc) {
    oracle_vjp_op(0, npe, n_elems, E, X, c, S, dX, dc);
}

/*
 * Elasticity (op 2): S [n_elems][nk(nk+1)/2] over the packed local DOF pairs,
 * c = (lambda, mu) per element, dc = (dL/dlambda, dL/dmu) per element (k_e is
 * linear in each), dX by the complex step of ke_elastic_z.
 */
static void elastic_vjp(int npe, int64_t n_elems, const int32_t *E, const double *X, const double *c,
                        const double *S, double *dX, double *dc) {
    const int nk = 3 * npe, np = nk * (nk + 1) / 2;
    double xe[24], ke[576];
    double complex xz[24], kz[576];
    for (int64_t e = 0; e < n_elems; ++e) {
        gather(npe, E, X, e, xe);
        for (int which = 0; which < 2; ++which) {
            ke_elastic(npe, xe, which == 0 ? 1.0 : 0.0, which == 1 ? 1.0 : 0.0, ke);
            double l1 = 0.0;
            for (int A = 0; A < nk; ++A)
                for (int B = 0; B <= A; ++B) l1 += S[e * np + A * (A + 1) / 2 + B] * ke[nk * A + B];
            dc[2 * e + which] = l1;
        }
        for (int k = 0; k < 3 * npe; ++k) {
            const double h = 1e-30 * (fabs(xe[k]) > 1.0 ? fabs(xe[k]) : 1.0);
            for (int m = 0; m < 3 * npe; ++m) xz[m] = xe[m];
            xz[k] += h * I;
            ke_elastic_z(npe, xz, c[2 * e], c[2 * e + 1], kz);
            double dl = 0.0;
            for (int A = 0; A < nk; ++A)
                for (int B = 0; B <= A; ++B) dl += S[e * np + A * (A + 1) / 2 + B] * cimag(kz[nk * A + B]) / h;
            dX[3 * (int64_t)E[e * npe + k / 3] + k % 3] += dl;
        }
    }
}
