/*
 * Plain FP64 CPU oracle for the closed-shell particle-particle ladder.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path and must never be used as a fallback for it.
 *
 * What it computes (the plain definition, no blocking, packing or symmetry):
 *
 *   Ladder term, Sec. "Acceleration of CC calculations", Eq. ppl-term with the
 *   Cholesky form of the integrals, Eq. cholesky, inserted (Eq. vfunction-chol):
 *
 *       R[i,j,a,b] += sum_{c,d} (ac|bd) t2[i,j,c,d],
 *       (ac|bd)     = sum_P L[P,a,c] L[P,b,d].
 *
 *   The einsum roles follow the paper's 'xac,xbd,icjd' labelling with the
 *   output ordered (i, j, a, b) and the amplitudes stored (i, j, c, d).
 *   The coefficient of the term is +1 and R is accumulated (R += ladder).
 *
 *   Ladder energy: E_L = sum_{ijab} (2 t2[i,j,a,b] - t2[i,j,b,a]) R[i,j,a,b],
 *   summed with Neumaier-compensated FP64 additions in (i, j, a, b) order.
 *
 * Summation orders (fixed, so results are reproducible bit for bit):
 *   V_ab[c,d]: P ascending, one rounded product and one rounded add per term.
 *   R[i,j,a,b]: a local sum over c ascending then d ascending, then one add
 *   into R.
 *
 * Compile without -ffast-math and with -ffp-contract=off so that no product
 * is fused into an FMA: every multiply and add is a separately rounded IEEE
 * FP64 operation on every host.
 *
 * Parity: pinned by the tests against numpy's einsum of the same definition,
 * exact integer arithmetic, closed forms (one Cholesky vector; one-hot
 * amplitudes), the R_ij^ab = R_ji^ba symmetry, linearity and an independent
 * trace formula for E_L.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX3(P, a, c, nv) (((size_t)(P) * (size_t)(nv) + (size_t)(a)) * (size_t)(nv) + (size_t)(c))
#define IDX4(i, j, a, b, no, nv) \
    ((((size_t)(i) * (size_t)(no) + (size_t)(j)) * (size_t)(nv) + (size_t)(a)) * (size_t)(nv) + (size_t)(b))

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* V_ab[c,d] = sum_P L[P,a,c] L[P,b,d]   (Eq. cholesky), P ascending. */
static void eri_pair(int nv, int nchol, const double* L, int a, int b, double* Vab) {
    for (size_t k = 0; k < (size_t)nv * nv; ++k) Vab[k] = 0.0;
    for (int P = 0; P < nchol; ++P) {
        const double* La = L + IDX3(P, a, 0, nv);
        const double* Lb = L + IDX3(P, b, 0, nv);
        for (int c = 0; c < nv; ++c) {
            const double lac = La[c];
            double* row = Vab + (size_t)c * nv;
            for (int d = 0; d < nv; ++d) row[d] += lac * Lb[d];
        }
    }
}

/* out[i,j] = sum_c sum_d V_ab[c,d] t2[i,j,c,d]  (Eq. ppl-term), c then d ascending. */
static void ladder_pair(int no, int nv, const double* Vab, const double* t2, double* out /* [no*no] */) {
    for (int i = 0; i < no; ++i) {
        for (int j = 0; j < no; ++j) {
            const double* tij = t2 + IDX4(i, j, 0, 0, no, nv);
            double s = 0.0;
            for (int c = 0; c < nv; ++c) {
                const double* vrow = Vab + (size_t)c * nv;
                const double* trow = tij + (size_t)c * nv;
                for (int d = 0; d < nv; ++d) s += vrow[d] * trow[d];
            }
            out[(size_t)i * no + j] = s;
        }
    }
}

/* R[i,j,a,b] += sum_{cd} (ac|bd) t2[i,j,c,d]  for all i, j, a, b.
 * Parallel over a; every R element is written by exactly one thread. */
int oracle_ladder(int no, int nv, int nchol, const double* L, const double* t2, double* R) {
    if (no <= 0 || nv <= 0 || nchol <= 0 || !L || !t2 || !R) return 1;
    int err = 0;
#pragma omp parallel
    {
        double* Vab = (double*)malloc(sizeof(double) * (size_t)nv * nv);
        double* tmp = (double*)malloc(sizeof(double) * (size_t)no * no);
        if (!Vab || !tmp) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int a = 0; a < nv; ++a) {
                for (int b = 0; b < nv; ++b) {
                    eri_pair(nv, nchol, L, a, b, Vab);
                    ladder_pair(no, nv, Vab, t2, tmp);
                    for (int i = 0; i < no; ++i)
                        for (int j = 0; j < no; ++j) R[IDX4(i, j, a, b, no, nv)] += tmp[(size_t)i * no + j];
                }
            }
        }
        free(Vab);
        free(tmp);
    }
    return err;
}

/* Row-subset mode: the ladder contribution (not accumulated) for the listed
 * (a, b) pairs, all (i, j):  out[k, i, j] = sum_{cd} (a_k c|b_k d) t2[i,j,c,d].
 * Uses exactly the loops of oracle_ladder, so its values are bit-identical to
 * the corresponding increments of the full mode. */
int oracle_ladder_pairs(int no, int nv, int nchol, const double* L, const double* t2, int npairs,
                        const int* a_list, const int* b_list, double* out) {
    if (no <= 0 || nv <= 0 || nchol <= 0 || npairs < 0 || !L || !t2 || (npairs && (!a_list || !b_list || !out)))
        return 1;
    for (int k = 0; k < npairs; ++k)
        if (a_list[k] < 0 || a_list[k] >= nv || b_list[k] < 0 || b_list[k] >= nv) return 1;
    int err = 0;
#pragma omp parallel
    {
        double* Vab = (double*)malloc(sizeof(double) * (size_t)nv * nv);
        if (!Vab) {
#pragma omp atomic write
            err = 2;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int k = 0; k < npairs; ++k) {
                eri_pair(nv, nchol, L, a_list[k], b_list[k], Vab);
                ladder_pair(no, nv, Vab, t2, out + (size_t)k * no * no);
            }
        }
        free(Vab);
    }
    return err;
}

/* Explicitly stored ERI block V[a,b,c,d] = (ac|bd) (Eq. cholesky), for small nv. */
int oracle_eri(int nv, int nchol, const double* L, double* V) {
    if (nv <= 0 || nchol <= 0 || !L || !V) return 1;
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) eri_pair(nv, nchol, L, a, b, V + ((size_t)a * nv + b) * nv * nv);
    return 0;
}

/* Ladder from a stored ERI block: R[i,j,a,b] += sum_{cd} V[a,b,c,d] t2[i,j,c,d]. */
int oracle_ladder_stored(int no, int nv, const double* V, const double* t2, double* R) {
    if (no <= 0 || nv <= 0 || !V || !t2 || !R) return 1;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)no * no);
    if (!tmp) return 2;
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b) {
            ladder_pair(no, nv, V + ((size_t)a * nv + b) * nv * nv, t2, tmp);
            for (int i = 0; i < no; ++i)
                for (int j = 0; j < no; ++j) R[IDX4(i, j, a, b, no, nv)] += tmp[(size_t)i * no + j];
        }
    free(tmp);
    return 0;
}

/* E_L = sum_{ijab} (2 t2[i,j,a,b] - t2[i,j,b,a]) R[i,j,a,b], Neumaier-compensated. */
double oracle_energy(int no, int nv, const double* t2, const double* R) {
    double sum = 0.0, comp = 0.0;
    for (int i = 0; i < no; ++i)
        for (int j = 0; j < no; ++j)
            for (int a = 0; a < nv; ++a)
                for (int b = 0; b < nv; ++b) {
                    const double u = 2.0 * t2[IDX4(i, j, a, b, no, nv)] - t2[IDX4(i, j, b, a, no, nv)];
                    const double term = u * R[IDX4(i, j, a, b, no, nv)];
                    const double s = sum + term;
                    if ((sum >= 0 ? sum : -sum) >= (term >= 0 ? term : -term))
                        comp += (sum - s) + term;
                    else
                        comp += (term - s) + sum;
                    sum = s;
                }
    return sum + comp;
}
