/*
 * FP64 CPU oracle for the alchemical nonbonded path of an absolute binding
 * free energy (ABFE) lambda window.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file. The product path never calls it, and it
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Every function is the plain definition written out in double precision:
 * all pairs, minimum image, hard cutoff, no neighbour list (except the cell
 * list used only by the self-check), no fusion or reordering. OpenMP only
 * splits independent rows; per-row partial sums are added in a fixed order, so
 * results do not depend on the thread count.
 *
 * Sources (the paper, "Development and large-scale benchmarks of a
 * protein-ligand absolute binding free energy toolkit"):
 *  - Beutler softcore LJ, Lorentz-Berthelot mixing, lambda_ij = min(l_i, l_j),
 *    alpha = 0.5, p = 1, softcore also between ligand atoms:
 *    section "Double annihilation protocol".
 *  - Ligand partial charges scaled linearly to zero with sterics on:
 *    section "Double annihilation protocol".
 *  - PME real-space cutoff 1.0 nm (the real-space erfc term only):
 *    appendix "Additional methodological details".
 *  - Boresch restraint: distance P1-L1, angles P1-L1-L2 and L1-P1-P2 with
 *    U = (k/2)(g-g0)^2, dihedrals P2-P1-L1-L2, P1-L1-L2-L3, L1-P1-P2-P3 with
 *    U = k[1 - cos(g-g0)]: section "Restraints".
 * Where the paper is silent this file reads it as follows: both LJ and the
 * erfc term are truncated hard at r < r_c with no switch, shift or dispersion
 * correction; the reciprocal-space, self and exclusion-correction terms of PME
 * are not part of this path, and excluded pairs contribute nothing; the
 * restraint enters as lambda_r * U_B (linear); ligand-ligand charge products
 * scale as lambda_q^2 (annihilation) or stay at full strength (decoupling).
 *
 * Parity status: every function here is pinned by tests in
 * tests/test_oracle_pins.py (closed forms, limits, finite differences,
 * brute force, published random-number test vectors).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t n;
    const double *pos;      /* [n][3] nm */
    const double *box;      /* [3] nm, orthorhombic */
    const double *charge;   /* [n] e */
    const double *sigma;    /* [n] nm */
    const double *epsilon;  /* [n] kJ/mol */
    const uint8_t *is_lig;  /* [n] 1 = alchemical ligand atom */
    const int32_t *ex_off;  /* [n+1] CSR offsets of excluded partners */
    const int32_t *ex_idx;  /* partners, both directions */
} orc_sys;

typedef struct {
    double cutoff;          /* r_c, nm */
    double beta;            /* Ewald splitting parameter, 1/nm */
    double alpha;           /* softcore alpha */
    double p;               /* softcore power p */
    double ke;              /* Coulomb constant, kJ mol^-1 nm e^-2 */
    int32_t mode;           /* 0 = annihilate (ligand-ligand scaled), 1 = decouple */
} orc_par;

/* Energy components, kJ/mol. */
enum { E_ENV_LJ = 0, E_ENV_C, E_LIGENV_LJ, E_LIGLIG_LJ, E_LIGENV_C, E_LIGLIG_C, E_N };

static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

static int excluded(const orc_sys *s, int i, int j) {
    for (int k = s->ex_off[i]; k < s->ex_off[i + 1]; ++k)
        if (s->ex_idx[k] == j) return 1;
    return 0;
}

/* One pair at separation r (r < r_c, not excluded).
 * out: comp = which energy slot each term goes to, u_lj, u_c, dU/dlambda_v,
 * dU/dlambda_q and fscal = -(dU/dr)/r. */
typedef struct { double u_lj, u_c, dudlv, dudlq, fscal; int slot_lj, slot_c; } pair_t;

static pair_t eval_pair(const orc_sys *s, const orc_par *P, int i, int j, double r2,
                        double lam_q, double lam_v) {
    pair_t o;
    const double r = sqrt(r2);
    const int li = s->is_lig[i], lj = s->is_lig[j];
    const int any = li || lj, both = li && lj;
    /* Lorentz-Berthelot mixing. */
    const double sig = 0.5 * (s->sigma[i] + s->sigma[j]);
    const double eps = sqrt(s->epsilon[i] * s->epsilon[j]);
    const double sig6 = sig * sig * sig * sig * sig * sig;
    /* lambda_ij = min(lambda_i, lambda_j), environment atoms at 1; in decouple
     * mode the ligand's own pairs stay at full coupling. */
    const int alch = any && !(both && P->mode == 1);
    o.u_lj = 0.0; o.dudlv = 0.0; o.dudlq = 0.0; o.fscal = 0.0;
    if (!alch) {
        const double sr6 = sig6 / (r2 * r2 * r2);
        o.u_lj = 4.0 * eps * (sr6 * sr6 - sr6);
        o.fscal = 4.0 * eps * (12.0 * sr6 * sr6 - 6.0 * sr6) / r2;
    } else {
        /* Beutler: r_eff^6 = alpha (1-lambda)^p sigma^6 + r^6,
         * U = lambda 4 eps (sigma^12 / r_eff^12 - sigma^6 / r_eff^6). */
        const double lam = lam_v;
        const double r6 = r2 * r2 * r2;
        const double s6 = P->alpha * pow(1.0 - lam, P->p) * sig6 + r6;
        const double a = sig6 * sig6 / (s6 * s6), b = sig6 / s6;
        const double g = 4.0 * eps * (a - b);                 /* unscaled energy */
        const double dg_ds = 4.0 * eps * (-2.0 * a + b) / s6;   /* d g / d s6 */
        o.u_lj = lam * g;
        /* dU/dr = lam dg/ds6 * 6 r^5  ->  fscal = -lam dg/ds6 * 6 r^4 */
        o.fscal = -lam * dg_ds * 6.0 * r2 * r2;
        /* dU/dlambda = g + lam dg/ds6 * ds6/dlambda, ds6/dlambda = -alpha p (1-lam)^(p-1) sigma^6 */
        const double ds_dl = -P->alpha * P->p * pow(1.0 - lam, P->p - 1.0) * sig6;
        o.dudlv = g + lam * dg_ds * ds_dl;
    }
    /* Real-space Ewald Coulomb with ligand charges scaled by lambda_q. */
    const double u1 = P->ke * s->charge[i] * s->charge[j] * erfc(P->beta * r) / r;
    const double f1 = P->ke * s->charge[i] * s->charge[j] *
                      (erfc(P->beta * r) / r + 2.0 * P->beta / sqrt(M_PI) *
                       exp(-P->beta * P->beta * r2)) / r2;
    double scale = 1.0, dscale = 0.0;
    if (any && !(both && P->mode == 1)) {
        if (both) { scale = lam_q * lam_q; dscale = 2.0 * lam_q; }
        else { scale = lam_q; dscale = 1.0; }
    }
    o.u_c = scale * u1;
    o.fscal += scale * f1;
    o.dudlq = dscale * u1;
    if (!any) { o.slot_lj = E_ENV_LJ; o.slot_c = E_ENV_C; }
    else if (both) { o.slot_lj = E_LIGLIG_LJ; o.slot_c = E_LIGLIG_C; }
    else { o.slot_lj = E_LIGENV_LJ; o.slot_c = E_LIGENV_C; }
    return o;
}

static void delta(const orc_sys *s, int i, int j, double d[3]) {
    for (int k = 0; k < 3; ++k)
        d[k] = min_image(s->pos[3 * j + k] - s->pos[3 * i + k], s->box[k]);
}

/*
 * Nonbonded energies, forces and lambda derivatives of one configuration at
 * (lam_q, lam_v). ligand_only = 1 restricts the sum to pairs with at least one
 * ligand atom (every pair whose energy depends on lambda). F may be NULL.
 * E[6] = {env LJ, env C, ligand-env LJ, ligand-ligand LJ, ligand-env C,
 * ligand-ligand C}; dudl[2] = {dU/dlambda_v, dU/dlambda_q};
 * npairs[2] = {env-env, ligand-involved} in-cutoff non-excluded pairs.
 */
int orc_nonbonded(const orc_sys *s, const orc_par *P, double lam_q, double lam_v,
                  int ligand_only, double *F, double *E, double *dudl, int64_t *npairs) {
    const int n = s->n;
    const double rc2 = P->cutoff * P->cutoff;
    const int NA = E_N + 4;  /* 6 energies, 2 derivatives, 2 counts (as doubles) */
    double *row = (double *)calloc((size_t)n * NA, sizeof(double));
    if (!row) return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < n; ++i) {
        if (ligand_only && !s->is_lig[i]) continue;
        double fi[3] = {0, 0, 0};
        double *acc = row + (size_t)i * NA;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            if (ligand_only && s->is_lig[j] && j < i) continue; /* each ligand pair once */
            double d[3];
            delta(s, i, j, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc2)) continue;
            if (excluded(s, i, j)) continue;
            pair_t o = eval_pair(s, P, i, j, r2, lam_q, lam_v);
            /* force on i is -fscal * (x_j - x_i) */
            for (int k = 0; k < 3; ++k) fi[k] -= o.fscal * d[k];
            const int count_here = ligand_only ? 1 : (j > i);
            if (count_here) {
                acc[o.slot_lj] += o.u_lj;
                acc[o.slot_c] += o.u_c;
                acc[E_N + 0] += o.dudlv;
                acc[E_N + 1] += o.dudlq;
                acc[E_N + ((s->is_lig[i] || s->is_lig[j]) ? 3 : 2)] += 1.0;
            }
        }
        if (F && !ligand_only)
            for (int k = 0; k < 3; ++k) F[3 * i + k] = fi[k];
    }
    double tot[10] = {0};
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < NA; ++a) tot[a] += row[(size_t)i * NA + a];
    free(row);
    if (E) for (int a = 0; a < E_N; ++a) E[a] = tot[a];
    if (dudl) { dudl[0] = tot[E_N]; dudl[1] = tot[E_N + 1]; }
    if (npairs) { npairs[0] = (int64_t)tot[E_N + 2]; npairs[1] = (int64_t)tot[E_N + 3]; }
    return 0;
}

/* Nonbonded force on each of the listed atoms (all partners), F[nrows][3]. */
int orc_force_rows(const orc_sys *s, const orc_par *P, double lam_q, double lam_v,
                   int nrows, const int32_t *rows, double *F) {
    const double rc2 = P->cutoff * P->cutoff;
#pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < nrows; ++r) {
        const int i = rows[r];
        double fi[3] = {0, 0, 0};
        for (int j = 0; j < s->n; ++j) {
            if (j == i) continue;
            double d[3];
            delta(s, i, j, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc2) || excluded(s, i, j)) continue;
            pair_t o = eval_pair(s, P, i, j, r2, lam_q, lam_v);
            for (int k = 0; k < 3; ++k) fi[k] -= o.fscal * d[k];
        }
        for (int k = 0; k < 3; ++k) F[3 * r + k] = fi[k];
    }
    return 0;
}

/* Number of in-cutoff non-excluded partners of each atom (all partners). */
int orc_neighbor_counts(const orc_sys *s, double rc, int32_t *count) {
    const double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < s->n; ++i) {
        int c = 0;
        for (int j = 0; j < s->n; ++j) {
            if (j == i) continue;
            double d[3];
            delta(s, i, j, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rc2 && !excluded(s, i, j)) ++c;
        }
        count[i] = c;
    }
    return 0;
}

/* All in-cutoff non-excluded pairs i<j by brute force, in (i, j) order. */
int64_t orc_pairs_brute(const orc_sys *s, double rc, int64_t cap, int32_t *out) {
    const double rc2 = rc * rc;
    int64_t m = 0;
    for (int i = 0; i < s->n; ++i)
        for (int j = i + 1; j < s->n; ++j) {
            double d[3];
            delta(s, i, j, d);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rc2 && !excluded(s, i, j)) {
                if (m < cap) { out[2 * m] = i; out[2 * m + 1] = j; }
                ++m;
            }
        }
    return m;
}

/*
 * The same pair set through a cell list (used only to check itself against
 * the brute-force set): cells at least r_c wide, each atom tested against the
 * atoms of the 27 surrounding cells, duplicates removed when a box has fewer
 * than three cells along an axis. Output is unordered; the caller sorts.
 */
int64_t orc_pairs_cell(const orc_sys *s, double rc, int64_t cap, int32_t *out) {
    int nc[3];
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int)floor(s->box[k] / rc);
        if (nc[k] < 1) nc[k] = 1;
    }
    const int ncell = nc[0] * nc[1] * nc[2];
    int *head = (int *)malloc(sizeof(int) * ncell);
    int *next = (int *)malloc(sizeof(int) * s->n);
    int *cell_of = (int *)malloc(sizeof(int) * s->n);
    if (!head || !next || !cell_of) { free(head); free(next); free(cell_of); return -1; }
    for (int c = 0; c < ncell; ++c) head[c] = -1;
    for (int i = s->n - 1; i >= 0; --i) {
        int ci[3];
        for (int k = 0; k < 3; ++k) {
            double x = s->pos[3 * i + k] - s->box[k] * floor(s->pos[3 * i + k] / s->box[k]);
            int c = (int)(x / s->box[k] * nc[k]);
            if (c >= nc[k]) c = nc[k] - 1;
            ci[k] = c;
        }
        const int c = (ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
        cell_of[i] = c;
        next[i] = head[c];
        head[c] = i;
    }
    const double rc2 = rc * rc;
    int64_t m = 0;
    for (int i = 0; i < s->n; ++i) {
        const int c = cell_of[i];
        const int cz = c % nc[2], cy = (c / nc[2]) % nc[1], cx = c / (nc[1] * nc[2]);
        int seen[27], nseen = 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    const int x = ((cx + dx) % nc[0] + nc[0]) % nc[0];
                    const int y = ((cy + dy) % nc[1] + nc[1]) % nc[1];
                    const int z = ((cz + dz) % nc[2] + nc[2]) % nc[2];
                    const int cc = (x * nc[1] + y) * nc[2] + z;
                    int dup = 0;
                    for (int t = 0; t < nseen; ++t) dup |= (seen[t] == cc);
                    if (dup) continue;
                    seen[nseen++] = cc;
                    for (int j = head[cc]; j >= 0; j = next[j]) {
                        if (j <= i) continue;
                        double d[3];
                        delta(s, i, j, d);
                        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 < rc2 && !excluded(s, i, j)) {
                            if (m < cap) { out[2 * m] = i; out[2 * m + 1] = j; }
                            ++m;
                        }
                    }
                }
    }
    free(head); free(next); free(cell_of);
    return m;
}

/* ------------------------------------------------------------------ restraint */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Angle at vertex b of a-b-c and its gradient with respect to a, b, c. */
static double angle_grad(const double *u /* a - b */, const double *v /* c - b */,
                         double ga[3], double gb[3], double gc[3]) {
    const double lu = sqrt(dot3(u, u)), lv = sqrt(dot3(v, v));
    double c = dot3(u, v) / (lu * lv);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    const double th = acos(c);
    const double sn = sqrt(1.0 - c * c);
    /* d(cos)/du = (v/|v| - cos u/|u|)/|u|; d(theta) = -d(cos)/sin */
    for (int k = 0; k < 3; ++k) {
        const double dcu = (v[k] / lv - c * u[k] / lu) / lu;
        const double dcv = (u[k] / lu - c * v[k] / lv) / lv;
        ga[k] = -dcu / sn;
        gc[k] = -dcv / sn;
        gb[k] = -(ga[k] + gc[k]);
    }
    return th;
}

/* Dihedral a-b-c-d, IUPAC sign: phi = atan2(|b2| b1.(b2 x b3), (b1 x b2).(b2 x b3)),
 * with b1 = b - a, b2 = c - b, b3 = d - c; gradient per atom. */
static double dihedral_grad(const double *b1, const double *b2, const double *b3,
                            double ga[3], double gb[3], double gc[3], double gd[3]) {
    double n1[3], n2[3];
    cross3(b1, b2, n1);
    cross3(b2, b3, n2);
    const double lb2 = sqrt(dot3(b2, b2));
    const double y = lb2 * dot3(b1, n2), x = dot3(n1, n2);
    const double phi = atan2(y, x);
    const double n1s = dot3(n1, n1), n2s = dot3(n2, n2);
    const double p = dot3(b1, b2) / (lb2 * lb2), q = dot3(b3, b2) / (lb2 * lb2);
    for (int k = 0; k < 3; ++k) {
        ga[k] = -lb2 / n1s * n1[k];
        gd[k] = lb2 / n2s * n2[k];
    }
    /* inner atoms (p, q are the projections of b1 and b3 on b2, in units of |b2|^2) */
    for (int k = 0; k < 3; ++k) {
        gb[k] = -(1.0 + p) * ga[k] + q * gd[k];
        gc[k] = p * ga[k] - (1.0 + q) * gd[k];
    }
    return phi;
}

static void mi_vec(const double *pos, const double *box, int from, int to, double *d) {
    for (int k = 0; k < 3; ++k) d[k] = min_image(pos[3 * to + k] - pos[3 * from + k], box[k]);
}

/*
 * Boresch restraint. anchors = (P1, P2, P3, L1, L2, L3). U_B is the unscaled
 * restraint energy (= dU/dlambda_r for U = lambda_r U_B); F (may be NULL) gets
 * lambda_r * (-grad U_B) added. geom[6] (may be NULL) receives
 * (r, theta_A, theta_B, phi_A, phi_B, phi_C).
 */
int orc_boresch(const double *pos, const double *box, const int32_t *anc, double r0,
                const double *theta0, const double *phi0, double kr, double kth, double kph,
                double lam_r, double *F, double *U_B, double *geom) {
    const int P1 = anc[0], P2 = anc[1], P3 = anc[2], L1 = anc[3], L2 = anc[4], L3 = anc[5];
    double g[6][3];          /* gradient of U_B with respect to P1 P2 P3 L1 L2 L3 */
    memset(g, 0, sizeof(g));
    double U = 0.0;
    double gm[6];
    /* distance P1-L1 */
    {
        double d[3];
        mi_vec(pos, box, P1, L1, d);
        const double r = sqrt(dot3(d, d));
        U += 0.5 * kr * (r - r0) * (r - r0);
        const double dU = kr * (r - r0);
        for (int k = 0; k < 3; ++k) { g[3][k] += dU * d[k] / r; g[0][k] -= dU * d[k] / r; }
        gm[0] = r;
    }
    /* angle P1-L1-L2 (vertex L1) */
    {
        double u[3], v[3], ga[3], gb[3], gc[3];
        mi_vec(pos, box, L1, P1, u);
        mi_vec(pos, box, L1, L2, v);
        const double th = angle_grad(u, v, ga, gb, gc);
        U += 0.5 * kth * (th - theta0[0]) * (th - theta0[0]);
        const double dU = kth * (th - theta0[0]);
        for (int k = 0; k < 3; ++k) { g[0][k] += dU * ga[k]; g[3][k] += dU * gb[k]; g[4][k] += dU * gc[k]; }
        gm[1] = th;
    }
    /* angle L1-P1-P2 (vertex P1) */
    {
        double u[3], v[3], ga[3], gb[3], gc[3];
        mi_vec(pos, box, P1, L1, u);
        mi_vec(pos, box, P1, P2, v);
        const double th = angle_grad(u, v, ga, gb, gc);
        U += 0.5 * kth * (th - theta0[1]) * (th - theta0[1]);
        const double dU = kth * (th - theta0[1]);
        for (int k = 0; k < 3; ++k) { g[3][k] += dU * ga[k]; g[0][k] += dU * gb[k]; g[1][k] += dU * gc[k]; }
        gm[2] = th;
    }
    /* dihedrals: (P2,P1,L1,L2), (P1,L1,L2,L3), (L1,P1,P2,P3) as anchor slots */
    const int dh[3][4] = {{1, 0, 3, 4}, {0, 3, 4, 5}, {3, 0, 1, 2}};
    for (int t = 0; t < 3; ++t) {
        const int a = anc[dh[t][0]], b = anc[dh[t][1]], c = anc[dh[t][2]], d = anc[dh[t][3]];
        double b1[3], b2[3], b3[3], ga[3], gb[3], gc[3], gd[3];
        mi_vec(pos, box, a, b, b1);
        mi_vec(pos, box, b, c, b2);
        mi_vec(pos, box, c, d, b3);
        const double phi = dihedral_grad(b1, b2, b3, ga, gb, gc, gd);
        U += kph * (1.0 - cos(phi - phi0[t]));
        const double dU = kph * sin(phi - phi0[t]);
        for (int k = 0; k < 3; ++k) {
            g[dh[t][0]][k] += dU * ga[k];
            g[dh[t][1]][k] += dU * gb[k];
            g[dh[t][2]][k] += dU * gc[k];
            g[dh[t][3]][k] += dU * gd[k];
        }
        gm[3 + t] = phi;
    }
    (void)P2; (void)P3; (void)L2; (void)L3;
    if (F)
        for (int s = 0; s < 6; ++s)
            for (int k = 0; k < 3; ++k) F[3 * anc[s] + k] -= lam_r * g[s][k];
    if (U_B) *U_B = U;
    if (geom) memcpy(geom, gm, sizeof(gm));
    return 0;
}

/* Harmonic bonds U = (k/2)(r - r0)^2 (minimum image); F (may be NULL) accumulates -grad U. */
int orc_bonds(const double *pos, const double *box, int nb, const int32_t *idx,
              const double *r0, const double *kb, double *F, double *U) {
    double u = 0.0;
    for (int b = 0; b < nb; ++b) {
        const int i = idx[2 * b], j = idx[2 * b + 1];
        double d[3];
        mi_vec(pos, box, i, j, d);
        const double r = sqrt(dot3(d, d));
        u += 0.5 * kb[b] * (r - r0[b]) * (r - r0[b]);
        if (F) {
            const double f = -kb[b] * (r - r0[b]) / r;   /* force on j along d */
            for (int k = 0; k < 3; ++k) { F[3 * j + k] += f * d[k]; F[3 * i + k] -= f * d[k]; }
        }
    }
    if (U) *U = u;
    return 0;
}

/* ------------------------------------------------------------------ random numbers */

/*
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit multiplications with
 * the published multipliers, a key bumped by the published Weyl constants.
 */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (r < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Three standard normal deviates per atom for one Langevin step, the counter
 * layout shared (by documentation, not code) with the CUDA integrator:
 * counter = (atom id, step low 32 bits, step high 32 bits, replica id),
 * key = (seed low 32 bits, seed high 32 bits). Uniforms u = (x + 0.5) / 2^32;
 * Box-Muller: z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1),
 * z2 = sqrt(-2 ln u2) cos(2 pi u3).
 */
void orc_gauss3(int n, uint64_t seed, uint64_t step, uint32_t replica, double *out) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int a = 0; a < n; ++a) {
        const uint32_t ctr[4] = {(uint32_t)a, (uint32_t)step, (uint32_t)(step >> 32), replica};
        uint32_t x[4];
        orc_philox4x32_10(ctr, key, x);
        double u[4];
        for (int k = 0; k < 4; ++k) u[k] = ((double)x[k] + 0.5) * (1.0 / 4294967296.0);
        const double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
        out[3 * a + 0] = r0 * cos(2.0 * M_PI * u[1]);
        out[3 * a + 1] = r0 * sin(2.0 * M_PI * u[1]);
        out[3 * a + 2] = r1 * cos(2.0 * M_PI * u[3]);
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
