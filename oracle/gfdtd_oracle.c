/*
 * gfdtd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU implementation of the generalized FDTD scheme of
 * Deck-Leger, Bahrami, Li and Caloz, "Generalized FDTD Scheme for the
 * Simulation of Electromagnetic Scattering in Moving Structures"
 * (arXiv 2304.06586).  It exists to check the CUDA library; only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header or constant with the CUDA path.
 *
 * What it computes (normalised units c = eps0 = mu0 = 1, so v = beta, and the
 * cell size dz = 1, the time step dt = S):
 *
 *   Moving perturbation (Sec. 4, Eqs. Farad_discr, Ampere_discr,
 *   Dconst_discr, Bconst_discr with the dynamic terms of Table 1):
 *     E*_k^{n-1/2}   = D_k^{n-1/2} / eps_k^{n-1/2} - beta * Bbar_k
 *                      Bbar_k = (B_{k-1/2} + B_{k-3/2})/2  for beta >= 0 (Table 1, Ba)
 *                             = (B_{k+3/2} + B_{k+1/2})/2  for beta <  0 (Table 1, Bb)
 *                      with B at level n-1
 *     B_{k+1/2}^n    = B^{n-1} - S (E*_{k+1} - E*_k) - beta S dB
 *                      dB = B_{k+1/2} - B_{k-1/2} (beta >= 0, Table 1 dBa)
 *                         = B_{k+3/2} - B_{k+1/2} (beta <  0, Table 1 dBb), level n-1
 *     H*_{k+1/2}^n   = B^n / mu^n - beta (D_{k+1} + D_k)^{n-1/2} / 2   (Table 1, Da = Db)
 *     D_k^{n+1/2}    = D^{n-1/2} - S (H*_{k+1/2} - H*_{k-1/2}) - beta S dD
 *                      dD = D_k - D_{k-1} (beta >= 0, Table 1 dDa)
 *                         = D_{k+1} - D_k (beta <  0, Table 1 dDb), level n-1/2
 *
 *   Moving matter (the paper derives the scheme for moving perturbation
 *   only; the moving-matter case changes the constitutive relations): with the
 *   footnote tensors of Eq. const_3d_regular in Eq. const_3d, the 1D star
 *   relations are eps' E* = (1 - beta^2) D - beta H* and
 *   mu' H* = (1 - beta^2) B - beta E*.  Solved for E* and H*:
 *     E* = D / eps_m - beta_c B,   H* = B / mu_m - beta_c D,
 *     1/eps_m = (1-beta^2) mu' / (n'^2 - beta^2),
 *     1/mu_m  = (1-beta^2) eps' / (n'^2 - beta^2),
 *     beta_c  = beta (1 - beta^2) / (n'^2 - beta^2),  n'^2 = eps' mu'.
 *   These have the moving-perturbation form, so they are discretized exactly
 *   like Eqs. Dconst_discr / Bconst_discr with the Table 1 averages (beta_c in
 *   place of beta in the averaged terms; beta itself in the upwind terms).  In
 *   moving vacuum (eps' = mu' = 1) beta_c = beta and 1/eps_m = 1/mu_m = 1, so
 *   the update is the moving-perturbation update.
 *
 *   Grid: D and E* live at integer nodes k in [0, nz); B and H* at k+1/2,
 *   stored at array index k.  The state between steps is (B^n, D^{n+1/2}).
 *   Every field outside [0, nz) is zero (the paper is silent on domain ends).
 *
 *   Material: eps and mu are sampled at the node's moving-frame coordinate
 *   xi = z - beta t (Eq. const_3d_regular: eps(r - v t)).  The coordinate is
 *   evaluated exactly in 32.32 fixed point: positions are integers in units of
 *   2^-32 cell, the profile breakpoints are rounded to that grid, and the
 *   displacement per half time step is dq = round(beta*S * 2^31).  A node at
 *   position p (k*2^32 for D, k*2^32 + 2^31 for B) at half level h (time
 *   h*S/2) has xi = p - dq*h.  Layers are half-open [z_{i-1}, z_i).
 *
 *   Source (Eq. spectrum_incident, real carrier): after the D update of step n,
 *     D_ks += amp * sin(w0 (t - t0)) * exp(-((t - t0)/tau)^2),  t = (n + 1/2) S.
 *
 *   Absorbing layers (the paper is silent on domain ends; an option of this
 *   library, not of the paper): with width W > 0, a field sample at position
 *   x (D_k at x = k, B_k at x = k + 1/2) is multiplied right after its update
 *   by g(x) = exp(-sigma d(x)^2), d = (W - x)/W for x < W, d = (x - (nz-1-W))/W
 *   for x > nz-1-W, else 0; the source is added after the D damping.
 *
 *   One-way (total-field / scattered-field) source (the paper is silent on
 *   sources beyond the soft one; an option of this library): a boundary at
 *   node q splits the grid into the total-field region (D_k, B_k with k >= q)
 *   and the scattered-field region (k < q).  The incident wave is the
 *   right-going wave that a soft source with the given waveform emits in an
 *   auxiliary grid of the same scheme filled with the uniform background (the
 *   material at node q at t = 0): graded absorbing layers of AUX_W = 512
 *   cells and strength 0.05 at both ends of an undamped interior of 40 cells
 *   (one carrier wavelength of the workloads), AUX_N = 1064 cells in all; the
 *   soft source 8 cells into the interior (aux node 520) and the boundary 12
 *   cells right of it (aux node 532; aux index = k - q + 532).  The width is
 *   set by an accuracy criterion: 512 is the smallest power of two for which
 *   the layers (strength 0.05 or 0.1) reflect less than 1e-6 of the incident
 *   amplitude in moving vacuum for |beta| <= 0.6 and less than 3e-6 in every
 *   stable uniform background with n|beta| <= 0.6, for a 40-cell carrier
 *   with 3- and 10-period envelopes (256 cells reflect up to 1.5e-6 in
 *   vacuum).  What the layers reflect reaches the scattered-field region.
 *   Every update that reads a value across the boundary reads it in the
 *   other region's convention: a total-field update adds the incident value
 *   of a scattered-field input, a scattered-field update subtracts the
 *   incident value of a total-field input.  Worked out on the stencil
 *   above (hb = beta_c / 2, ie = 1/eps_m, im = 1/mu_m of the background;
 *   Bi, Di the incident B^{n-1}, D^{n-1/2}, Bn the incident B^n), this adds
 *   after the B update
 *     beta >= 0: B_{q-1} += S ie Di_q,
 *                B_q     += -S hb Bi_{q-2} + beta S Bi_{q-1},
 *                B_{q+1} += -S hb Bi_{q-1};
 *     beta <  0: B_{q-2} += -S hb Bi_q,
 *                B_{q-1} += S ie Di_q - S hb Bi_{q+1} + beta S Bi_q;
 *   and after the D update
 *     D_{q-1} += -S hb Di_q  (+ beta S Di_q when beta < 0),
 *     D_q     += S (im Bn_{q-1} - hb Di_{q-1})  (+ beta S Di_{q-1} when beta >= 0).
 *   Outside the auxiliary grid's reach (q - 2 .. q + 1) nothing changes.
 *
 *   Probes: F = E at the probe node at level n+1/2 (moving perturbation:
 *   E = D/eps exactly, Eq. const_1d; moving matter: E = E* + beta * Bbar with
 *   E* from the relation above and Bbar the Table 1 average of B^n), and for
 *   every bin
 *     X(w) += F * exp(+i w t) * dt,   t = (n + 1/2) S,  dt = S.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t kind;        /* 0: moving perturbation, 1: moving matter */
    int32_t interp;      /* 0: layers (piecewise constant), 1: piecewise linear */
    int32_t n;           /* number of layers (interp 0) or knots (interp 1) */
    int32_t reserved;
    const double* z;     /* interp 0: n-1 boundaries; interp 1: n knots; cells, moving frame, t = 0 */
    const double* eps;   /* n values (relative permittivity; eps' at rest for matter) */
    const double* mu;    /* n values */
    double beta;         /* v / c */
    double S;            /* Courant number dt/dz */
    int64_t nz;          /* cells */
    int64_t absorb_width;  /* cells of the graded absorbing layer at each end (0: none) */
    double absorb_sigma;   /* its strength at the outer end */
} orc_problem;

typedef struct {
    int64_t node;
    double omega0, tau, t0, amp;
} orc_source;

typedef struct {
    int64_t node;        /* q: first node of the total-field region */
    double omega0, tau, t0, amp;   /* waveform of the auxiliary soft source */
    double* aux_B;       /* AUX_N doubles: auxiliary state (caller-owned, zero at the start) */
    double* aux_D;
} orc_tfsf;

#define AUX_N 1064
#define AUX_W 512
#define AUX_SRC 520
#define AUX_Q 532

typedef struct {
    int64_t node;
    int32_t n_bins;
    int32_t reserved;
    const double* omega; /* n_bins angular frequencies */
    double* re;          /* n_bins accumulators (in/out) */
    double* im;
    double* series;      /* optional: F per step of this call (length n_steps) */
} orc_probe;

/* ---- material sampling (exact fixed-point moving coordinate) ------------ */

typedef struct {
    int n, interp;
    int64_t* zq;
    const double* val;
} orc_profile;

static int64_t to_fixed(double x) { return llround(ldexp(x, 32)); }

/* index of the last breakpoint <= xi, or -1 (binary search over sorted zq) */
static int last_at_or_below(const int64_t* zq, int m, int64_t xi)
{
    int lo = -1, hi = m;                 /* invariant: zq[lo] <= xi < zq[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (zq[mid] <= xi) lo = mid; else hi = mid;
    }
    return lo;
}

static double profile_at(const orc_profile* pr, int64_t xi)
{
    if (pr->interp == 0) {
        /* value i holds on [z_{i-1}, z_i): i = number of boundaries <= xi */
        int i = last_at_or_below(pr->zq, pr->n - 1, xi) + 1;
        return pr->val[i];
    }
    if (xi <= pr->zq[0]) return pr->val[0];
    if (xi >= pr->zq[pr->n - 1]) return pr->val[pr->n - 1];
    int i = last_at_or_below(pr->zq, pr->n, xi);
    double w = (double)(xi - pr->zq[i]) / (double)(pr->zq[i + 1] - pr->zq[i]);
    return pr->val[i] + w * (pr->val[i + 1] - pr->val[i]);
}

/* position of integer node k and of half node k+1/2, in units of 2^-32 cell */
static int64_t node_pos(int64_t k) { return k * 4294967296LL; }
static int64_t half_pos(int64_t k) { return k * 4294967296LL + 2147483648LL; }

/* ---- helpers: fields outside [0, nz) are zero ---------------------------- */

static double at(const double* a, int64_t i, int64_t nz) { return (i < 0 || i >= nz) ? 0.0 : a[i]; }

static double source_value(const orc_source* s, double t)
{
    double u = t - s->t0;
    return s->amp * sin(s->omega0 * u) * exp(-(u / s->tau) * (u / s->tau));
}

/* E* from D and the averaged B (perturbation: Eq. Dconst_discr; matter: the
   solved star relation), and H* from B and the averaged D (Eq. Bconst_discr). */
static double estar(int kind, double beta, double e, double m, double d, double bbar)
{
    if (kind == 0) return d / e - beta * bbar;
    double den = e * m - beta * beta;
    double g = 1.0 - beta * beta;
    return g * m / den * d - beta * g / den * bbar;
}

static double hstar(int kind, double beta, double e, double m, double b, double dbar)
{
    if (kind == 0) return b / m - beta * dbar;
    double den = e * m - beta * beta;
    double g = 1.0 - beta * beta;
    return g * e / den * b - beta * g / den * dbar;
}

/* ---- absorbing layers ------------------------------------------------------ */

/* damping factor of a field sample at position x (cells) */
static double absorb_factor(const orc_problem* p, double x)
{
    const double W = (double)p->absorb_width;
    double d = 0.0;
    if (x < W) d = (W - x) / W;
    else if (x > (double)(p->nz - 1) - W) d = (x - ((double)(p->nz - 1) - W)) / W;
    return exp(-p->absorb_sigma * d * d);
}

/* ---- the time loop ------------------------------------------------------- */

int orc_run_tfsf(const orc_problem* p, int n_src, const orc_source* src,
                 int n_probe, orc_probe* probes, int n_tfsf, const orc_tfsf* tfsf,
                 int64_t n_done, int64_t n_steps, double* B, double* D);

/* The auxiliary problem of a one-way source: the background material of node
   q at t = 0, uniform, with the same kind, velocity and Courant number. */
static void tfsf_aux_problem(const orc_problem* p, const orc_profile* eps, const orc_profile* mu,
                             int64_t q, double* e_bg, double* m_bg, orc_problem* aux)
{
    *e_bg = profile_at(eps, node_pos(q));
    *m_bg = profile_at(mu, node_pos(q));
    memset(aux, 0, sizeof(*aux));
    aux->kind = p->kind;
    aux->interp = 0;
    aux->n = 1;
    aux->z = NULL;
    aux->eps = e_bg;
    aux->mu = m_bg;
    aux->beta = p->beta;
    aux->S = p->S;
    aux->nz = AUX_N;
    aux->absorb_width = AUX_W;
    aux->absorb_sigma = 0.05;
}

int orc_run(const orc_problem* p, int n_src, const orc_source* src,
            int n_probe, orc_probe* probes,
            int64_t n_done, int64_t n_steps,
            double* B, double* D)
{
    return orc_run_tfsf(p, n_src, src, n_probe, probes, 0, NULL, n_done, n_steps, B, D);
}

int orc_run_tfsf(const orc_problem* p, int n_src, const orc_source* src,
                 int n_probe, orc_probe* probes, int n_tfsf, const orc_tfsf* tfsf,
                 int64_t n_done, int64_t n_steps, double* B, double* D)
{
    const int64_t nz = p->nz;
    const double beta = p->beta, S = p->S;
    const int pos = beta >= 0.0;
    if (nz <= 0 || p->n < 1 || (p->interp == 1 && p->n < 2)) return -1;

    int nb = p->interp == 0 ? p->n - 1 : p->n;
    orc_profile eps = {p->n, p->interp, NULL, p->eps};
    orc_profile mu = {p->n, p->interp, NULL, p->mu};
    int64_t* zq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    for (int i = 0; i < nb; ++i) zq[i] = to_fixed(p->z[i]);
    eps.zq = zq;
    mu.zq = zq;
    const int64_t dq = llround(ldexp(beta * S, 31));   /* beta*S/2 cells per half step */

    /* one-way sources: auxiliary problems, background coefficients, per-step corrections */
    const int nt = n_tfsf > 0 ? n_tfsf : 0;
    orc_problem* aux = (orc_problem*)malloc(sizeof(orc_problem) * (size_t)(nt + 1));
    double* bg = (double*)malloc(sizeof(double) * (size_t)(2 * nt + 1));   /* eps, mu per source */
    double* corr = (double*)malloc(sizeof(double) * (size_t)(6 * nt + 1));  /* dB q-2..q+1, dD q-1..q */
    for (int i = 0; i < nt; ++i) tfsf_aux_problem(p, &eps, &mu, tfsf[i].node, &bg[2 * i], &bg[2 * i + 1], &aux[i]);

    double* Es = (double*)malloc(sizeof(double) * (size_t)nz);  /* E* (perturbation: recomputed) */
    double* Hs = (double*)malloc(sizeof(double) * (size_t)nz);  /* H* */
    double* Bo = (double*)malloc(sizeof(double) * (size_t)nz);  /* B^{n-1} */
    double* Do = (double*)malloc(sizeof(double) * (size_t)nz);  /* D^{n-1/2} */

    for (int64_t s = 0; s < n_steps; ++s) {
        const int64_t n = n_done + s + 1;      /* B^{n-1} -> B^n, D^{n-1/2} -> D^{n+1/2} */
        memcpy(Bo, B, sizeof(double) * (size_t)nz);
        memcpy(Do, D, sizeof(double) * (size_t)nz);

        /* one-way sources: incident values before and after the auxiliary step */
        for (int i = 0; i < nt; ++i) {
            const int64_t q = tfsf[i].node, a = AUX_Q - q;   /* aux index = k + a */
            double* aB = tfsf[i].aux_B;
            double* aD = tfsf[i].aux_D;
            const double Bim2 = aB[q - 2 + a], Bim1 = aB[q - 1 + a], Bi0 = aB[q + a], Bip1 = aB[q + 1 + a];
            const double Dim1 = aD[q - 1 + a], Di0 = aD[q + a];
            orc_source as = {AUX_SRC, tfsf[i].omega0, tfsf[i].tau, tfsf[i].t0, tfsf[i].amp};
            orc_run_tfsf(&aux[i], 1, &as, 0, NULL, 0, NULL, n - 1, 1, aB, aD);
            const double Bn_m1 = aB[q - 1 + a];
            const double e = bg[2 * i], m = bg[2 * i + 1];
            double ie, im, bc;
            if (p->kind == 0) {
                ie = 1.0 / e; im = 1.0 / m; bc = beta;
            } else {
                const double den = e * m - beta * beta, g = 1.0 - beta * beta;
                ie = g * m / den; im = g * e / den; bc = beta * g / den;
            }
            const double hb = 0.5 * bc;
            double* c = &corr[6 * i];
            if (pos) {
                c[0] = 0.0;
                c[1] = S * ie * Di0;
                c[2] = -S * hb * Bim2 + beta * S * Bim1;
                c[3] = -S * hb * Bim1;
                c[4] = -S * hb * Di0;
                c[5] = S * (im * Bn_m1 - hb * Dim1) + beta * S * Dim1;
            } else {
                c[0] = -S * hb * Bi0;
                c[1] = S * ie * Di0 - S * hb * Bip1 + beta * S * Bi0;
                c[2] = 0.0;
                c[3] = 0.0;
                c[4] = -S * hb * Di0 + beta * S * Di0;
                c[5] = S * (im * Bn_m1 - hb * Dim1);
            }
        }

        /* E*^{n-1/2} (Eq. Dconst_discr with Table 1 Ba/Bb, B at level n-1) */
        for (int64_t k = 0; k < nz; ++k) {
            double e = profile_at(&eps, node_pos(k) - dq * (2 * n - 1));
            double m = profile_at(&mu, node_pos(k) - dq * (2 * n - 1));
            double bbar = pos ? 0.5 * (at(Bo, k - 1, nz) + at(Bo, k - 2, nz))
                              : 0.5 * (at(Bo, k + 1, nz) + at(Bo, k, nz));
            Es[k] = estar(p->kind, beta, e, m, Do[k], bbar);
        }

        /* B^n (Eq. Farad_discr with Table 1 dBa/dBb) */
        for (int64_t k = 0; k < nz; ++k) {
            double dB = pos ? Bo[k] - at(Bo, k - 1, nz) : at(Bo, k + 1, nz) - Bo[k];
            B[k] = Bo[k] - S * (at(Es, k + 1, nz) - Es[k]) - beta * S * dB;
        }
        if (p->absorb_width > 0)
            for (int64_t k = 0; k < nz; ++k) B[k] *= absorb_factor(p, (double)k + 0.5);
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < 4; ++j) {
                const int64_t k = tfsf[i].node - 2 + j;
                if (k >= 0 && k < nz) B[k] += corr[6 * i + j];
            }

        /* H*^n (Eq. Bconst_discr with Table 1 Da/Db, D at level n-1/2) */
        for (int64_t k = 0; k < nz; ++k) {
            double e = profile_at(&eps, half_pos(k) - dq * (2 * n));
            double m = profile_at(&mu, half_pos(k) - dq * (2 * n));
            double dbar = 0.5 * (Do[k] + at(Do, k + 1, nz));
            Hs[k] = hstar(p->kind, beta, e, m, B[k], dbar);
        }

        /* D^{n+1/2} (Eq. Ampere_discr with Table 1 dDa/dDb) */
        for (int64_t k = 0; k < nz; ++k) {
            double dD = pos ? Do[k] - at(Do, k - 1, nz) : at(Do, k + 1, nz) - Do[k];
            D[k] = Do[k] - S * (Hs[k] - at(Hs, k - 1, nz)) - beta * S * dD;
        }
        if (p->absorb_width > 0)
            for (int64_t k = 0; k < nz; ++k) D[k] *= absorb_factor(p, (double)k);
        for (int i = 0; i < nt; ++i)
            for (int j = 0; j < 2; ++j) {
                const int64_t k = tfsf[i].node - 1 + j;
                if (k >= 0 && k < nz) D[k] += corr[6 * i + 4 + j];
            }

        /* soft source at t_{n+1/2} */
        const double t = (double)(2 * n + 1) * S * 0.5;
        for (int i = 0; i < n_src; ++i) {
            if (src[i].node >= 0 && src[i].node < nz) D[src[i].node] += source_value(&src[i], t);
        }

        /* probes: physical E at level n+1/2, running DFT */
        for (int i = 0; i < n_probe; ++i) {
            int64_t k = probes[i].node;
            if (k < 0 || k >= nz) continue;
            double e = profile_at(&eps, node_pos(k) - dq * (2 * n + 1));
            double F;
            if (p->kind == 0) {
                F = D[k] / e;                       /* Eq. const_1d: D = eps E */
            } else {
                double m = profile_at(&mu, node_pos(k) - dq * (2 * n + 1));
                double bbar = pos ? 0.5 * (at(B, k - 1, nz) + at(B, k - 2, nz))
                                  : 0.5 * (at(B, k + 1, nz) + at(B, k, nz));
                F = estar(1, beta, e, m, D[k], bbar) + beta * bbar;   /* E = E* + v B */
            }
            if (probes[i].series) probes[i].series[s] = F;
            for (int f = 0; f < probes[i].n_bins; ++f) {
                double w = probes[i].omega[f];
                probes[i].re[f] += F * cos(w * t) * S;
                probes[i].im[f] += F * sin(w * t) * S;
            }
        }
    }
    free(zq); free(Es); free(Hs); free(Bo); free(Do); free(aux); free(bg); free(corr);
    return 0;
}

/* eps (or mu, which = 1) sampled at every integer node (which = 0) or half
   node (which = 1) at half level h: the same material rule the time loop uses. */
int orc_sample_material(const orc_problem* p, int which_field, int half_node, int64_t h, double* out)
{
    int nb = p->interp == 0 ? p->n - 1 : p->n;
    int64_t* zq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    for (int i = 0; i < nb; ++i) zq[i] = to_fixed(p->z[i]);
    orc_profile pr = {p->n, p->interp, zq, which_field == 0 ? p->eps : p->mu};
    const int64_t dq = llround(ldexp(p->beta * p->S, 31));
    for (int64_t k = 0; k < p->nz; ++k) {
        int64_t x = half_node ? half_pos(k) : node_pos(k);
        out[k] = profile_at(&pr, x - dq * h);
    }
    free(zq);
    return 0;
}

/* ---- discrete adjoint (moving perturbation) ------------------------------
 *
 * The forward step n is linear in (B, D):
 *   E_k  = D_k/eps_k - beta bbar_k(B)                 (level n-1/2)
 *   B'_k = B_k - S (E_{k+1} - E_k) - beta S dB_k(B)
 *   H_k  = B'_k/mu_k - beta (D_k + D_{k+1})/2          (level n)
 *   D'_k = D_k - S (H_k - H_{k-1}) - beta S dD_k(D)
 * (the source adds a constant).  orc_step_transpose applies the transpose of
 * this map, operation by operation in reverse order, to adjoint fields
 * (aB', aD') and returns (aB, aD); it also adds dL/deps_k at level n-1/2,
 * i.e. aE_k * (-D_k / eps_k^2), into geps[k].  Indices outside [0, nz) are
 * absent, exactly as the forward map's zero ghost fields.
 */
int orc_step_transpose(const orc_problem* p, int64_t n, const double* aBn, const double* aDn,
                       const double* D_old, double* aB, double* aD, double* geps)
{
    const int64_t nz = p->nz;
    const double beta = p->beta, S = p->S;
    const int pos = beta >= 0.0;
    if (p->kind != 0 || p->absorb_width > 0) return -1;   /* no transpose of the absorber here */
    int nb = p->interp == 0 ? p->n - 1 : p->n;
    int64_t* zq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    for (int i = 0; i < nb; ++i) zq[i] = to_fixed(p->z[i]);
    orc_profile eps = {p->n, p->interp, zq, p->eps};
    orc_profile mu = {p->n, p->interp, zq, p->mu};
    const int64_t dq = llround(ldexp(beta * S, 31));
    double* aH = (double*)calloc((size_t)nz, sizeof(double));
    double* aBp = (double*)calloc((size_t)nz, sizeof(double));
    double* aE = (double*)calloc((size_t)nz, sizeof(double));
    for (int64_t k = 0; k < nz; ++k) { aB[k] = 0.0; aD[k] = 0.0; aBp[k] = aBn[k]; }

    /* D'_k = D_k - S (H_k - H_{k-1}) - beta S dD_k(D) */
    for (int64_t k = 0; k < nz; ++k) {
        aD[k] += aDn[k];
        aH[k] += -S * aDn[k];
        if (k - 1 >= 0) aH[k - 1] += S * aDn[k];
        if (pos) {                 /* dD_k = D_k - D_{k-1} */
            aD[k] += -beta * S * aDn[k];
            if (k - 1 >= 0) aD[k - 1] += beta * S * aDn[k];
        } else {                   /* dD_k = D_{k+1} - D_k */
            if (k + 1 < nz) aD[k + 1] += -beta * S * aDn[k];
            aD[k] += beta * S * aDn[k];
        }
    }
    /* H_k = B'_k/mu_k - beta (D_k + D_{k+1})/2 */
    for (int64_t k = 0; k < nz; ++k) {
        double m = profile_at(&mu, half_pos(k) - dq * (2 * n));
        aBp[k] += aH[k] / m;
        aD[k] += -0.5 * beta * aH[k];
        if (k + 1 < nz) aD[k + 1] += -0.5 * beta * aH[k];
    }
    /* B'_k = B_k - S (E_{k+1} - E_k) - beta S dB_k(B) */
    for (int64_t k = 0; k < nz; ++k) {
        aB[k] += aBp[k];
        aE[k] += S * aBp[k];
        if (k + 1 < nz) aE[k + 1] += -S * aBp[k];
        if (pos) {                 /* dB_k = B_k - B_{k-1} */
            aB[k] += -beta * S * aBp[k];
            if (k - 1 >= 0) aB[k - 1] += beta * S * aBp[k];
        } else {                   /* dB_k = B_{k+1} - B_k */
            if (k + 1 < nz) aB[k + 1] += -beta * S * aBp[k];
            aB[k] += beta * S * aBp[k];
        }
    }
    /* E_k = D_k/eps_k - beta bbar_k(B) */
    for (int64_t k = 0; k < nz; ++k) {
        double e = profile_at(&eps, node_pos(k) - dq * (2 * n - 1));
        aD[k] += aE[k] / e;
        if (geps) geps[k] += aE[k] * (-D_old[k] / (e * e));
        if (pos) {                 /* bbar_k = (B_{k-1} + B_{k-2})/2 */
            if (k - 1 >= 0) aB[k - 1] += -0.5 * beta * aE[k];
            if (k - 2 >= 0) aB[k - 2] += -0.5 * beta * aE[k];
        } else {                   /* bbar_k = (B_{k+1} + B_k)/2 */
            if (k + 1 < nz) aB[k + 1] += -0.5 * beta * aE[k];
            aB[k] += -0.5 * beta * aE[k];
        }
    }
    free(aH); free(aBp); free(aE); free(zq);
    return 0;
}

/* Add g * d eps(xi)/d value_i for the node at moving coordinate xi into grad[i]. */
static void scatter_eps_grad(const orc_profile* pr, int64_t xi, double g, double* grad)
{
    if (pr->interp == 0) {
        grad[last_at_or_below(pr->zq, pr->n - 1, xi) + 1] += g;
        return;
    }
    if (xi <= pr->zq[0]) { grad[0] += g; return; }
    if (xi >= pr->zq[pr->n - 1]) { grad[pr->n - 1] += g; return; }
    int i = last_at_or_below(pr->zq, pr->n, xi);
    double w = (double)(xi - pr->zq[i]) / (double)(pr->zq[i + 1] - pr->zq[i]);
    grad[i] += g * (1.0 - w);
    grad[i + 1] += g * w;
}

/* Loss and gradient.  From the state (B0, D0) at step n0, runs n_steps forward
 * steps storing D after every step, forms L = sum_f |X_f|^2 of the probe's
 * bins (X accumulated over these steps only, as in orc_run), then sweeps back
 * with orc_step_transpose and returns dL/d(eps value i) of the profile in
 * grad[0..n). */
int orc_adjoint(const orc_problem* p, int n_src, const orc_source* src, const orc_probe* probe,
                int64_t n0, int64_t n_steps, const double* B0, const double* D0,
                double* loss, double* grad)
{
    const int64_t nz = p->nz;
    const double S = p->S;
    if (p->kind != 0 || p->absorb_width > 0 || n_steps < 1) return -1;
    double* Dh = (double*)malloc(sizeof(double) * (size_t)nz * (size_t)(n_steps + 1));
    double* B = (double*)malloc(sizeof(double) * (size_t)nz);
    double* series = (double*)malloc(sizeof(double) * (size_t)n_steps);
    double* re = (double*)calloc((size_t)probe->n_bins, sizeof(double));
    double* im = (double*)calloc((size_t)probe->n_bins, sizeof(double));
    memcpy(B, B0, sizeof(double) * (size_t)nz);
    memcpy(Dh, D0, sizeof(double) * (size_t)nz);
    orc_probe pr = *probe;
    pr.re = re; pr.im = im; pr.series = NULL;
    for (int64_t s = 0; s < n_steps; ++s) {
        double* Dn = Dh + (size_t)(s + 1) * (size_t)nz;
        memcpy(Dn, Dh + (size_t)s * (size_t)nz, sizeof(double) * (size_t)nz);
        pr.series = series + s;
        orc_run(p, n_src, src, 1, &pr, n0 + s, 1, B, Dn);
    }
    double L = 0.0;
    for (int f = 0; f < probe->n_bins; ++f) L += re[f] * re[f] + im[f] * im[f];
    *loss = L;

    int nb = p->interp == 0 ? p->n - 1 : p->n;
    int64_t* zq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb > 0 ? nb : 1));
    for (int i = 0; i < nb; ++i) zq[i] = to_fixed(p->z[i]);
    orc_profile eps = {p->n, p->interp, zq, p->eps};
    const int64_t dq = llround(ldexp(p->beta * S, 31));
    for (int i = 0; i < p->n; ++i) grad[i] = 0.0;
    double* aB = (double*)calloc((size_t)nz, sizeof(double));
    double* aD = (double*)calloc((size_t)nz, sizeof(double));
    double* aB0 = (double*)calloc((size_t)nz, sizeof(double));
    double* aD0 = (double*)calloc((size_t)nz, sizeof(double));
    double* geps = (double*)calloc((size_t)nz, sizeof(double));
    const int64_t kp = probe->node;
    for (int64_t s = n_steps - 1; s >= 0; --s) {
        const int64_t n = n0 + s + 1;
        const double t = (double)(2 * n + 1) * S * 0.5;
        /* dL/dF_n = 2 S sum_f (Re X_f cos(w t) + Im X_f sin(w t)) */
        double g = 0.0;
        for (int f = 0; f < probe->n_bins; ++f) {
            double w = probe->omega[f];
            g += 2.0 * S * (re[f] * cos(w * t) + im[f] * sin(w * t));
        }
        const double* Dn = Dh + (size_t)(s + 1) * (size_t)nz;
        if (kp >= 0 && kp < nz) {
            /* F_n = D_kp / eps_kp (level n+1/2) */
            double e = profile_at(&eps, node_pos(kp) - dq * (2 * n + 1));
            aD[kp] += g / e;
            scatter_eps_grad(&eps, node_pos(kp) - dq * (2 * n + 1), g * (-Dn[kp] / (e * e)), grad);
        }
        for (int64_t k = 0; k < nz; ++k) geps[k] = 0.0;
        orc_step_transpose(p, n, aB, aD, Dh + (size_t)s * (size_t)nz, aB0, aD0, geps);
        for (int64_t k = 0; k < nz; ++k)
            if (geps[k] != 0.0) scatter_eps_grad(&eps, node_pos(k) - dq * (2 * n - 1), geps[k], grad);
        memcpy(aB, aB0, sizeof(double) * (size_t)nz);
        memcpy(aD, aD0, sizeof(double) * (size_t)nz);
    }
    free(Dh); free(B); free(series); free(re); free(im); free(zq);
    free(aB); free(aD); free(aB0); free(aD0); free(geps);
    return 0;
}

/* ---- 2D TE generalized scheme (test infrastructure) ----------------------
 *
 * Sec. 3 and Sec. 4 before the 1D reduction, for moving perturbation in the
 * x-z plane (d/dy = 0), motion along z, the TE polarisation E = E_y y^,
 * B = (B_x, 0, B_z), D = D_y y^, H = (H_x, 0, H_z):
 *   Eq. star:        E*_y = E_y + v B_x,   H*_x = H_x + v D_y,   H*_z = H_z
 *                    (v x B = v B_x y^,  v x D = -v D_y x^)
 *   Eq. const_3d:    D_y = eps (E*_y - v B_x),  B_x = mu (H*_x - v D_y),
 *                    B_z = mu H*_z
 *   Eq. Maxwell_star with curl(v x B) = -v dB/dz (v uniform, div B = 0) and
 *   curl(v x D) = -v dD/dz (div D = 0):
 *     dB_x/dt =  dE*_y/dz - v dB_x/dz
 *     dB_z/dt = -dE*_y/dx - v dB_z/dz
 *     dD_y/dt =  dH*_x/dz - dH*_z/dx - v dD_y/dz
 * Along z the terms are discretized exactly as the 1D scheme (Table 1: the
 * average of B_x in E*_y, the average of D_y in H*_x, the upwind differences
 * of every component); along x they are the standard Yee differences.  With
 * b = -B_x the z-part is the 1D update of Eqs. Farad_discr .. Bconst_discr.
 *
 * Grid (dz = 1, dx given, S = dt/dz, Sx = dt/dx): D_y at (i, k), B_x at
 * (i, k+1/2), B_z at (i+1/2, k); arrays [i * nz + k].  Periodic in x (nx
 * columns), every field zero outside [0, nz) in z.  Medium: layers of the
 * moving coordinate xi = z - v t - slope x (boundary b at xi = z_b, slanted
 * when slope != 0), evaluated exactly in 32.32 fixed point: a node at (x, z)
 * at half level h has xi = z 2^32 - dq h - round(x slope 2^32), dq as in 1D.
 * Soft line source: D_y(i, ks) += amp s(t) cos(kx i dx), s as in 1D.
 * Probes: E_y = D_y / eps at node (i, k), running DFT as in 1D.
 */
typedef struct {
    int64_t nx, nz;
    double dx, S, beta, slope;
    int32_t n, reserved;
    const double* z;      /* n-1 boundaries (moving frame, t = 0, at x = 0) */
    const double* eps;
    const double* mu;
} orc2_problem;

typedef struct {
    int64_t k;            /* z node of the line source */
    double kx;            /* transverse wavenumber of its cos(kx x) weight */
    double omega0, tau, t0, amp;
} orc2_source;

typedef struct {
    int64_t i, k;
    int32_t n_bins, reserved;
    const double* omega;
    double* re;
    double* im;
} orc2_probe;

static double orc2_material(const orc2_problem* p, const int64_t* zq, const double* val,
                            double x, int64_t zpos, int64_t dq, int64_t h)
{
    const int64_t xi = zpos - dq * h - llround(ldexp(x * p->slope, 32));
    int i = last_at_or_below(zq, p->n - 1, xi) + 1;
    return val[i];
}

static double at2(const double* a, int64_t nx, int64_t nz, int64_t i, int64_t k)
{
    if (k < 0 || k >= nz) return 0.0;
    i = ((i % nx) + nx) % nx;
    return a[i * nz + k];
}

int orc2_run(const orc2_problem* p, int n_src, const orc2_source* src, int n_probe, orc2_probe* probes,
             int64_t n_done, int64_t n_steps, double* Bx, double* Bz, double* D)
{
    const int64_t nx = p->nx, nz = p->nz, N = nx * nz;
    const double beta = p->beta, S = p->S, Sx = p->S / p->dx;
    const int pos = beta >= 0.0;
    if (nx < 1 || nz < 1 || p->n < 1 || !(p->dx > 0.0)) return -1;
    int64_t* zq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(p->n > 1 ? p->n - 1 : 1));
    for (int i = 0; i + 1 < p->n; ++i) zq[i] = to_fixed(p->z[i]);
    const int64_t dq = llround(ldexp(beta * S, 31));
    double* Es = (double*)malloc(sizeof(double) * (size_t)N);
    double* Hx = (double*)malloc(sizeof(double) * (size_t)N);
    double* Hz = (double*)malloc(sizeof(double) * (size_t)N);
    double* Bxo = (double*)malloc(sizeof(double) * (size_t)N);
    double* Bzo = (double*)malloc(sizeof(double) * (size_t)N);
    double* Do = (double*)malloc(sizeof(double) * (size_t)N);
    for (int64_t s = 0; s < n_steps; ++s) {
        const int64_t n = n_done + s + 1;
        memcpy(Bxo, Bx, sizeof(double) * (size_t)N);
        memcpy(Bzo, Bz, sizeof(double) * (size_t)N);
        memcpy(Do, D, sizeof(double) * (size_t)N);
        /* E*_y^{n-1/2} = D/eps + v Bbar_x (Table 1 Ba/Bb along z, B_x at level n-1) */
        for (int64_t i = 0; i < nx; ++i)
            for (int64_t k = 0; k < nz; ++k) {
                const double e = orc2_material(p, zq, p->eps, (double)i * p->dx, node_pos(k), dq, 2 * n - 1);
                const double bbar = pos ? 0.5 * (at2(Bxo, nx, nz, i, k - 1) + at2(Bxo, nx, nz, i, k - 2))
                                        : 0.5 * (at2(Bxo, nx, nz, i, k + 1) + at2(Bxo, nx, nz, i, k));
                Es[i * nz + k] = Do[i * nz + k] / e + beta * bbar;
            }
        /* B_x^n, B_z^n */
        for (int64_t i = 0; i < nx; ++i)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = i * nz + k;
                const double dbx = pos ? Bxo[c] - at2(Bxo, nx, nz, i, k - 1) : at2(Bxo, nx, nz, i, k + 1) - Bxo[c];
                Bx[c] = Bxo[c] + S * (at2(Es, nx, nz, i, k + 1) - Es[c]) - beta * S * dbx;
                const double dbz = pos ? Bzo[c] - at2(Bzo, nx, nz, i, k - 1) : at2(Bzo, nx, nz, i, k + 1) - Bzo[c];
                Bz[c] = Bzo[c] - Sx * (at2(Es, nx, nz, i + 1, k) - Es[c]) - beta * S * dbz;
            }
        /* H*_x^n = B_x/mu + v Dbar (Table 1 Da/Db, D at level n-1/2); H*_z^n = B_z/mu */
        for (int64_t i = 0; i < nx; ++i)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = i * nz + k;
                const double mx = orc2_material(p, zq, p->mu, (double)i * p->dx, half_pos(k), dq, 2 * n);
                const double mz = orc2_material(p, zq, p->mu, ((double)i + 0.5) * p->dx, node_pos(k), dq, 2 * n);
                const double dbar = 0.5 * (Do[c] + at2(Do, nx, nz, i, k + 1));
                Hx[c] = Bx[c] / mx + beta * dbar;
                Hz[c] = Bz[c] / mz;
            }
        /* D_y^{n+1/2} */
        for (int64_t i = 0; i < nx; ++i)
            for (int64_t k = 0; k < nz; ++k) {
                const int64_t c = i * nz + k;
                const double dd = pos ? Do[c] - at2(Do, nx, nz, i, k - 1) : at2(Do, nx, nz, i, k + 1) - Do[c];
                D[c] = Do[c] + S * (Hx[c] - at2(Hx, nx, nz, i, k - 1)) - Sx * (Hz[c] - at2(Hz, nx, nz, i - 1, k))
                       - beta * S * dd;
            }
        /* line sources at t_{n+1/2} */
        const double t = (double)(2 * n + 1) * S * 0.5;
        for (int q = 0; q < n_src; ++q) {
            if (src[q].k < 0 || src[q].k >= nz) continue;
            const double u = t - src[q].t0;
            const double sv = src[q].amp * sin(src[q].omega0 * u) * exp(-(u / src[q].tau) * (u / src[q].tau));
            for (int64_t i = 0; i < nx; ++i) D[i * nz + src[q].k] += sv * cos(src[q].kx * (double)i * p->dx);
        }
        /* probes: E_y = D_y / eps at level n+1/2 */
        for (int q = 0; q < n_probe; ++q) {
            const int64_t i = probes[q].i, k = probes[q].k;
            if (i < 0 || i >= nx || k < 0 || k >= nz) continue;
            const double e = orc2_material(p, zq, p->eps, (double)i * p->dx, node_pos(k), dq, 2 * n + 1);
            const double F = D[i * nz + k] / e;
            for (int f = 0; f < probes[q].n_bins; ++f) {
                const double w = probes[q].omega[f];
                probes[q].re[f] += F * cos(w * t) * S;
                probes[q].im[f] += F * sin(w * t) * S;
            }
        }
    }
    free(zq); free(Es); free(Hx); free(Hz); free(Bxo); free(Bzo); free(Do);
    return 0;
}
