/*
 * CP-factor FP64 oracle for GridWorld MDPs (test infrastructure only: used
 * by the tests, the smoke check and the CPU baseline of the benchmark; the
 * CUDA library never links it and it includes nothing of the library).
 *
 * The transition model of action a is the sum of its rank-1 terms
 * (CP form, background section and Fig. 1): each term moves one coordinate
 * by -1, 0 or +1 and leaves the others unchanged (identity factors on the
 * other dimensions), with weight lambda:
 *   intended move along the action's axis ............ lambda = p
 *   each of the 2(D-1) perpendicular unit moves ........ lambda = (1-p)/(2(D-1))
 *   D = 1 only: stay in place ........................... lambda = 1-p
 * A term whose move leaves the grid or enters an obstacle keeps the agent in
 * s (the obstacle correction that is not separable per dimension).
 *
 * The backup is Eq. 1, V'(s) = R(s) + gamma max_a sum_{s'} P(s'|s,a) V(s'),
 * evaluated term by term in plain loops: O(|S| x |C(s)| x |A|) work as in the
 * paper's complexity section. Terminal states keep V = R(t) (the interaction
 * ends), obstacles are not states (V = 0, policy 255).
 *
 * Parity pins: tests/test_oracle_pins.py compares every entry point with the
 * tabular definitions on small grids and with closed forms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { CELL_FREE = 0, CELL_OBSTACLE = 1, CELL_TERMINAL = 2 };
#define MAXD 16

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Rank-1 terms of action a: returns the count, fills dim/step/weight. */
static int action_terms(int D, int a, double p, int *dim, int *step, double *w) {
    int d = a / 2, sigma = (a % 2) ? 1 : -1, n = 0;
    dim[n] = d; step[n] = sigma; w[n] = p; n++;
    if (D == 1) {
        dim[n] = d; step[n] = 0; w[n] = 1.0 - p; n++;
    } else {
        double q = (1.0 - p) / (2.0 * (D - 1));
        for (int d2 = 0; d2 < D; d2++) {
            if (d2 == d) continue;
            dim[n] = d2; step[n] = -1; w[n] = q; n++;
            dim[n] = d2; step[n] = +1; w[n] = q; n++;
        }
    }
    return n;
}

/* Q(s, a) = R(s) + gamma * E_a[V](s) for a free state s with coordinates c. */
static double q_value(int D, const int64_t *shape, const int64_t *stride, double p, double gamma,
                      const uint8_t *cell, const double *R, const double *V,
                      int64_t s, const int64_t *c, int a) {
    int dim[2 * MAXD], step[2 * MAXD];
    double w[2 * MAXD];
    int nt = action_terms(D, a, p, dim, step, w);
    double e = 0.0;
    for (int t = 0; t < nt; t++) {
        int64_t x = c[dim[t]] + step[t];
        int64_t target = s;
        if (x >= 0 && x < shape[dim[t]]) {
            target = s + (int64_t)step[t] * stride[dim[t]];
            if (cell && cell[target] == CELL_OBSTACLE) target = s;
        }
        e += w[t] * V[target];
    }
    return R[s] + gamma * e;
}

/*
 * One synchronous backup over all states.
 *   fixed_pi == NULL : value-iteration backup (max over actions, Eq. 1);
 *   fixed_pi != NULL : policy-evaluation backup with the action fixed.
 * pi_out (may be NULL) receives the greedy action (lowest index on ties),
 * or fixed_pi's action; 255 on obstacles and terminals.
 * Q_out (may be NULL) receives Q[a * S + s] for free states, 0 elsewhere.
 * Returns max |V' - V| over non-obstacle states.
 */
double oracle_gw_backup(int D, const int64_t *shape, double p, double gamma,
                        const uint8_t *cell, const double *R, const double *V, double *Vout,
                        const uint8_t *fixed_pi, uint8_t *pi_out, double *Q_out) {
    int64_t S = 1, stride[MAXD];
    for (int d = D - 1; d >= 0; d--) { stride[d] = S; S *= shape[d]; }
    int A = 2 * D;
    double res = 0.0;
#pragma omp parallel for schedule(static) reduction(max : res)
    for (int64_t s = 0; s < S; s++) {
        uint8_t kind = cell ? cell[s] : CELL_FREE;
        if (kind != CELL_FREE) {
            double v = (kind == CELL_TERMINAL) ? R[s] : 0.0;
            Vout[s] = v;
            if (pi_out) pi_out[s] = 255;
            if (Q_out) for (int a = 0; a < A; a++) Q_out[(int64_t)a * S + s] = 0.0;
            if (kind == CELL_TERMINAL) {
                double dv = fabs(v - V[s]);
                if (dv > res) res = dv;
            }
            continue;
        }
        int64_t c[MAXD], rem = s;
        for (int d = 0; d < D; d++) { c[d] = rem / stride[d]; rem -= c[d] * stride[d]; }
        double best = -INFINITY;
        int arg = 0;
        if (fixed_pi) {
            arg = fixed_pi[s];
            best = q_value(D, shape, stride, p, gamma, cell, R, V, s, c, arg);
            if (Q_out) Q_out[(int64_t)arg * S + s] = best;
        } else {
            for (int a = 0; a < A; a++) {
                double q = q_value(D, shape, stride, p, gamma, cell, R, V, s, c, a);
                if (Q_out) Q_out[(int64_t)a * S + s] = q;
                if (q > best) { best = q; arg = a; }
            }
        }
        Vout[s] = best;
        if (pi_out) pi_out[s] = (uint8_t)arg;
        double dv = fabs(best - V[s]);
        if (dv > res) res = dv;
    }
    return res;
}

/*
 * Value iteration (background section): repeat the backup from V (in/out)
 * until max |V' - V| < tol or max_iter sweeps. pi_out gets the policy that
 * is greedy with respect to the returned V. Returns the sweep count, or -1
 * when out of memory. *res_out receives the last residual.
 */
int oracle_gw_value_iteration(int D, const int64_t *shape, double p, double gamma,
                              const uint8_t *cell, const double *R, double *V, uint8_t *pi_out,
                              double tol, int max_iter, double *res_out) {
    int64_t S = 1;
    for (int d = 0; d < D; d++) S *= shape[d];
    double *W = (double *)malloc((size_t)S * sizeof(double));
    if (!W) return -1;
    double res = INFINITY;
    int k = 0;
    double *cur = V, *nxt = W;
    while (k < max_iter) {
        res = oracle_gw_backup(D, shape, p, gamma, cell, R, cur, nxt, NULL, NULL, NULL);
        double *t = cur; cur = nxt; nxt = t;
        k++;
        if (res < tol) break;
    }
    if (cur != V) memcpy(V, cur, (size_t)S * sizeof(double));
    if (pi_out) oracle_gw_backup(D, shape, p, gamma, cell, R, V, W, NULL, pi_out, NULL);
    free(W);
    if (res_out) *res_out = res;
    return k;
}

/*
 * Iterative policy evaluation for the fixed policy pi (the evaluation step
 * of policy iteration), from V (in/out) until max |V' - V| < tol or
 * max_iter sweeps. Returns the sweep count, or -1 when out of memory.
 */
int oracle_gw_evaluate(int D, const int64_t *shape, double p, double gamma,
                       const uint8_t *cell, const double *R, const uint8_t *pi, double *V,
                       double tol, int max_iter, double *res_out) {
    int64_t S = 1;
    for (int d = 0; d < D; d++) S *= shape[d];
    double *W = (double *)malloc((size_t)S * sizeof(double));
    if (!W) return -1;
    double res = INFINITY;
    int k = 0;
    double *cur = V, *nxt = W;
    while (k < max_iter) {
        res = oracle_gw_backup(D, shape, p, gamma, cell, R, cur, nxt, pi, NULL, NULL);
        double *t = cur; cur = nxt; nxt = t;
        k++;
        if (res < tol) break;
    }
    if (cur != V) memcpy(V, cur, (size_t)S * sizeof(double));
    free(W);
    if (res_out) *res_out = res;
    return k;
}

/*
 * Q(s, a) for a list of states only (sampled checks at sizes where a full
 * sweep is too slow): Q_out[i * A + a] for states[i]; obstacles and
 * terminals get 0. Returns 0.
 */
int oracle_gw_q_states(int D, const int64_t *shape, double p, double gamma, const uint8_t *cell,
                       const double *R, const double *V, const int64_t *states, int64_t n,
                       double *Q_out) {
    int64_t S = 1, stride[MAXD];
    for (int d = D - 1; d >= 0; d--) { stride[d] = S; S *= shape[d]; }
    int A = 2 * D;
    for (int64_t i = 0; i < n; i++) {
        int64_t s = states[i];
        uint8_t kind = cell ? cell[s] : CELL_FREE;
        for (int a = 0; a < A; a++) Q_out[i * A + a] = 0.0;
        if (kind != CELL_FREE) continue;
        int64_t c[MAXD], rem = s;
        for (int d = 0; d < D; d++) { c[d] = rem / stride[d]; rem -= c[d] * stride[d]; }
        for (int a = 0; a < A; a++) Q_out[i * A + a] = q_value(D, shape, stride, p, gamma, cell, R, V, s, c, a);
    }
    return 0;
}
