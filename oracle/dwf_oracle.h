/*
 * dwf_oracle.h -- plain FP64 CPU oracle for the domain-wall operator and solver of
 * Chiu, Hsieh, Mao, Ogawa, "GPU-Based Conjugate Gradient Solver for Lattice QCD
 * with Domain-Wall Fermions" (Lattice 2010).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA path.
 *
 * Conventions (fixed readings of what the paper leaves open):
 *   dims = {Nx, Ny, Nz, Nt}, all even; mu = 0,1,2,3 for x,y,z,t; periodic
 *   boundaries.  Site index x + Nx*(y + Ny*(z + Nz*t)) (Sec. 3.1), parity
 *   (x+y+z+t) mod 2.  s is 0-based here (1-based in Eq. 4).
 *   5D spinor host layout (Sec. 3.1): complex index ((site*Ns + s)*4 + spin)*3 + colour,
 *   i.e. real index c + 24 s + 24 Ns site with c = reim + 2 (colour + 3 spin).
 *   Gauge field: complex index ((site*4 + mu)*3 + a)*3 + b, U_mu(x)_{ab}.
 *   Gamma matrices: chiral basis gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
 *   gamma_4 = [[0,1],[1,0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.
 *   Ns x Ns matrices are row-major, M[s*Ns + s'].
 *
 * Every function returns 0 on success, -1 on invalid arguments.
 */
#ifndef DWF_ORACLE_H
#define DWF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* gamma matrix mu (0..3 = x,y,z,t; 4 = gamma_5) as 4x4 complex, row-major, re/im interleaved */
int or_gamma(int mu, double *out32);

/* Wilson operator of Eq. 2 (d = 4, with the (d - m0) term) on every s-slice of a 5D field. */
int or_dw(const int dims[4], int Ns, const double *U, double m0, const double *in, double *out);

/* Hopping block of Eq. 12: out(x) = D^{p,1-p} in for the sites x of parity p;
 * sites of the other parity in out are set to 0. */
int or_hop(const int dims[4], int Ns, const double *U, int p, const double *in, double *out);

/* Literal adjoint of or_hop's block: out = (D^{p,1-p})^dagger in; in lives on parity p,
 * out on parity 1-p (sites of parity p in out are set to 0). */
int or_hop_dag(const int dims[4], int Ns, const double *U, int p, const double *in, double *out);

/* The chiral hopping matrices of Eq. 3-4: Lp = L_+, Lm = L_- = L_+^T (Ns x Ns). */
int or_lmat(int Ns, double m0, double mq, double *Lp, double *Lm);

/* M5 of Eq. 8 (second form) for each chirality, by Gauss-Jordan inversion. */
int or_m5(int Ns, double m0, double mq, const double *omega, const double *sigma,
          double *M5p, double *M5m);

/* S1 = M5 omega^{-1/2} and S2 = Y^{-1} sqrt(omega) of Eq. 9, per chirality. */
int or_s1s2(int Ns, double m0, double mq, const double *omega, const double *sigma,
            double *S1p, double *S1m, double *S2p, double *S2m);

/* u_s = sum_s' M_{ss'} v_s' with Mp on spins 0,1 (P+) and Mm on spins 2,3 (P-).
 * transpose != 0 uses M^T.  parity < 0: all sites; else only sites of that parity
 * (the others are set to 0). */
int or_apply_s(const int dims[4], int Ns, const double *Mp, const double *Mm, int transpose,
               int parity, const double *in, double *out);

/* Full 5D operator of Eq. 1 on the whole lattice. */
int or_dfull(const int dims[4], int Ns, const double *U, double m0, double mq,
             const double *omega, const double *sigma, const double *in, double *out);

/* Schur complement of Eq. 11 on parity p: C = 1 - M5 D^{p,1-p} M5 D^{1-p,p}
 * (p = 1 is the paper's odd-site form).  in/out are full-lattice arrays; only
 * parity-p sites are read, the other sites of out are 0. */
int or_c(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m,
         int p, const double *in, double *out);
/* Literal adjoint of or_c. */
int or_cdag(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m,
            int p, const double *in, double *out);
/* C C^dagger */
int or_ccdag(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m,
             int p, const double *in, double *out);

/* Conjugate gradient (Algorithm 1) on A = C C^dagger of parity p, FP64.
 * x holds the initial guess on entry.  Stops when |r| <= tol |b| or after maxiter
 * iterations.  iters/relres (may be NULL) receive the count and the recomputed
 * true residual |b - A x| / |b|. */
int or_cg(const int dims[4], int Ns, const double *U, const double *M5p, const double *M5m,
          int p, const double *b, double *x, double tol, int maxiter, int *iters, double *relres);

/* Full solve D psi = eta through Eq. 10: eta' = S1 eta, b = eta'_p - M5 D^{p,1-p} eta'_{1-p},
 * C C^dagger y = b by CG, phi_p = C^dagger y, phi_{1-p} = eta'_{1-p} - M5 D^{1-p,p} phi_p,
 * psi = S2 phi. */
int or_solve_full(const int dims[4], int Ns, const double *U, double m0, double mq,
                  const double *omega, const double *sigma, int p, const double *eta,
                  double *psi, double tol, int maxiter, int *iters, double *relres);

/* Euclidean inner product <a, b> = sum conj(a) b over all components; re/im out. */
int or_dot(long nreal, const double *a, const double *b, double *re, double *im);

#ifdef __cplusplus
}
#endif
#endif
