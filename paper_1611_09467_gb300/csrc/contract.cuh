// Contraction programs of the PEPS sampling path as strided small GEMMs.
//
// Every tensor contraction of the path (zip-up row absorption, single-row and
// two-row transfer steps, site environment) is a product C = A * B whose
// row, column and reduction indices each group at most two tensor indices,
// plus an optional batch index.  A `GemmDesc` records, for each operand, how
// a flattened index maps to a memory offset; the builders below are the only
// place where index orders are spelled out, and they are __host__ __device__
// so the host-side executor (used by the CPU tests) runs exactly the same
// descriptors as the kernels.
//
// Padded layouts (all row-major):
//   site tensor T  [l][r][u][d]           D^4      (Eq. 1, A_i at fixed s_i)
//   MPS tensor  M  [a][p][b]              Dc*D*Dc  (boundary MPS, Fig. 1d)
//   1-row transfer F[a][l][a'] / G        Dc*D*Dc
//   2-row transfer E[a][l1][l2][a'] / H   Dc*D*D*Dc
#pragma once

#if defined(__CUDACC__)
#define PEPS_HD __host__ __device__ __forceinline__
#else
#define PEPS_HD inline
#endif

namespace peps {

// Flattened index x -> (x / n2) * s1 + (x % n2) * s2.
struct Ix {
  int n2, s1, s2;
};

PEPS_HD Ix ix1(int s) { return Ix{1 << 30, 0, s}; }
PEPS_HD Ix ix2(int n2, int s1, int s2) { return Ix{n2, s1, s2}; }
PEPS_HD int ixoff(const Ix& m, int x) { return (x / m.n2) * m.s1 + (x % m.n2) * m.s2; }

// C[b](i, j) (+)= sum_k A[b](i, k) * B[b](k, j).  The reduction index is split
// as k = k1 * kn2 + k2 with the same kn2 for A and B (ak.n2 == bk.n2 == kn2).
struct GemmDesc {
  int M, N, K, nb;        // sizes, batch count
  Ix am, ak, bk, bn, cm, cn;
  int sa, sb, sc;         // batch strides
};

PEPS_HD Ix kx(int kn2, int s1, int s2) { return Ix{kn2, s1, s2}; }

PEPS_HD GemmDesc gemm(int M, int N, int K, Ix am, Ix ak, Ix bk, Ix bn, Ix cm, Ix cn) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K; g.nb = 1;
  g.am = am; g.ak = ak; g.bk = bk; g.bn = bn; g.cm = cm; g.cn = cn;
  g.sa = g.sb = g.sc = 0;
  return g;
}

// ---------------------------------------------------------------- transfers
// Single-row left transfer (sandwich <U_{r-1}| row r |L_{r+1}>, column c):
//   F_c[b,r,b'] = sum F_{c-1}[a,l,a'] Mu[a,u,b] T[l,r,u,d] Md[a',d,b'].
//   s0: P[a'][b][l][u] = F . Mu   (sum a)
//   s1: Q[b][r][a'][d] = P . T    (sum l,u)
//   s2: F'[b][r][b']   = Q . Md   (sum a',d)
PEPS_HD GemmDesc col1_left_step(int s, int D, int Dc) {
  const int DD = D * D, D3 = D * D * D;
  switch (s) {
    case 0:
      return gemm(D * Dc, D * Dc, Dc,
                  ix1(1), kx(Dc, 0, D * Dc),                 // A = F[a][l][a']: rows (l,a'), k = a
                  kx(Dc, 0, D * Dc), ix1(1),                 // B = Mu[a][u][b]: cols (u,b)
                  ix2(Dc, D, Dc * DD), ix2(Dc, 1, DD));      // C = P[a'][b][l][u]
    case 1:
      return gemm(Dc * Dc, DD, DD,
                  ix1(DD), kx(D, D, 1),                      // A = P: rows (a',b), k = (l,u)
                  kx(D, D3, D), ix2(D, DD, 1),               // B = T[l][r][u][d]: k=(l,u), cols (r,d)
                  ix2(Dc, D, D * Dc * D), ix2(D, Dc * D, 1)); // C = Q[b][r][a'][d]
    default:
      return gemm(Dc * D, Dc, Dc * D,
                  ix1(Dc * D), kx(D, D, 1),                  // A = Q: rows (b,r), k = (a',d)
                  kx(D, D * Dc, Dc), ix1(1),                 // B = Md[a'][d][b']
                  ix1(Dc), ix1(1));                          // C = F'[b][r][b']
  }
}

// Single-row right transfer:
//   G_c[a,l,a'] = sum Mu[a,u,b] T[l,r,u,d] Md[a',d,b'] G_{c+1}[b,r,b'].
//   s0: P[a][b'][u][r] = Mu . G  (sum b)
//   s1: Q[a][l][d][b'] = P . T   (sum u,r)
//   s2: G'[a][l][a']   = Q . Md  (sum d,b')
PEPS_HD GemmDesc col1_right_step(int s, int D, int Dc) {
  const int DD = D * D, D3 = D * D * D;
  switch (s) {
    case 0:
      return gemm(Dc * D, D * Dc, Dc,
                  ix1(Dc), kx(Dc, 0, 1),                     // A = Mu: rows (a,u), k = b
                  kx(Dc, 0, D * Dc), ix1(1),                 // B = G[b][r][b']: cols (r,b')
                  ix2(D, Dc * DD, D), ix2(Dc, 1, DD));       // C = P[a][b'][u][r]
    case 1:
      return gemm(Dc * Dc, DD, DD,
                  ix1(DD), kx(D, D, 1),                      // A = P: rows (a,b'), k = (u,r)
                  kx(D, D, DD), ix2(D, D3, 1),               // B = T: k = (u,r), cols (l,d)
                  ix2(Dc, DD * Dc, 1), ix2(D, D * Dc, Dc));  // C = Q[a][l][d][b']
    default:
      return gemm(Dc * D, Dc, D * Dc,
                  ix1(D * Dc), kx(Dc, Dc, 1),                // A = Q: rows (a,l), k = (d,b')
                  kx(Dc, Dc, 1), ix1(D * Dc),                // B = Md[a'][d][b']: k = (d,b'), cols a'
                  ix1(Dc), ix1(1));                          // C = G'[a][l][a']
  }
}

// Site environment (the B of Delta = B / W):
//   B[l,r,u,d] = sum F[a,l,a'] Mu[a,u,b] Md[a',d,b'] G[b,r,b'].
//   s0: Z[a'][d][b][r]       = Md . G   (sum b')
//   s1: R[a][a'][u][d][r]    = Mu . Z   (sum b)
//   s2: B[l][r][u][d]        = F . R    (sum a,a')
PEPS_HD GemmDesc site_env_step(int s, int D, int Dc) {
  const int DD = D * D, D3 = D * D * D;
  switch (s) {
    case 0:
      return gemm(Dc * D, Dc * D, Dc,
                  ix1(Dc), kx(Dc, 0, 1),                     // A = Md: rows (a',d), k = b'
                  kx(Dc, 0, 1), ix1(Dc),                     // B = G[b][r][b']: cols (b,r)
                  ix1(Dc * D), ix1(1));                      // C = Z[a'][d][b][r]
    case 1:
      return gemm(Dc * D, Dc * DD, Dc,
                  ix1(Dc), kx(Dc, 0, 1),                     // A = Mu: rows (a,u), k = b
                  kx(Dc, 0, D), ix2(D, Dc * D, 1),           // B = Z: k = b, cols (a',d,r)
                  ix2(D, Dc * D3, DD), ix2(DD, D3, 1));      // C = R[a][a'][u][d][r]
    default:
      return gemm(D, D3, Dc * Dc,
                  ix1(Dc), kx(Dc, D * Dc, 1),                // A = F: rows l, k = (a,a')
                  kx(Dc, Dc * D3, D3), ix1(1),               // B = R: k = (a,a'), cols (u,d,r)
                  ix1(D3), ix2(D, 1, DD));                   // C = B[l][r][u][d]
  }
}

// Environment of the candidate tensor in the overlap <P| Mu T> (the
// variational-fit truncation): the single-row left transfer with the Md slot
// left open.
//   P[a',d,b'] = sum F[a,l,a'] Mu[a,u,b] T[l,r,u,d] G[b,r,b'].
//   s0, s1: as col1_left_step (P[a'][b][l][u], then Q[b][r][a'][d])
//   s2: P[a'][d][b'] = Q . G   (sum b,r)
PEPS_HD GemmDesc fit_site_step(int s, int D, int Dc) {
  if (s < 2) return col1_left_step(s, D, Dc);
  return gemm(Dc * D, Dc, Dc * D,
              ix1(1), kx(D, D * Dc * D, Dc * D),             // A = Q[b][r][a'][d]: rows (a',d), k = (b,r)
              kx(D, D * Dc, Dc), ix1(1),                     // B = G[b][r][b']: k = (b,r), cols b'
              ix1(Dc), ix1(1));                              // C = P[a'][d][b']
}

// Two-row left transfer (sandwich <U_{r-1}| rows r,r+1 |L_{r+2}>):
//   E_c[b,r1,r2,b'] = sum E_{c-1}[a,l1,l2,a'] Mu[a,u1,b] T1[l1,r1,u1,m] T2[l2,r2,m,d2] Md[a',d2,b'].
//   s0: P1[l2][a'][b][l1][u1]  = E . Mu   (sum a)
//   s1: P2[a'][b][r1][l2][m]   = P1 . T1  (sum l1,u1)
//   s2: P3[b][r1][r2][a'][d2]  = P2 . T2  (sum l2,m)
//   s3: E'[b][r1][r2][b']      = P3 . Md  (sum a',d2)
PEPS_HD GemmDesc col2_left_step(int s, int D, int Dc) {
  const int DD = D * D, D3 = D * D * D;
  switch (s) {
    case 0:
      return gemm(DD * Dc, D * Dc, Dc,
                  ix1(1), kx(Dc, 0, DD * Dc),                // A = E: rows (l1,l2,a'), k = a
                  kx(Dc, 0, D * Dc), ix1(1),                 // B = Mu: cols (u1,b)
                  ix2(D * Dc, D, Dc * DD), ix2(Dc, 1, DD));  // C = P1[l2][a'][b][l1][u1]
    case 1:
      return gemm(D * Dc * Dc, DD, DD,
                  ix1(DD), kx(D, D, 1),                      // A = P1: rows (l2,a',b), k = (l1,u1)
                  kx(D, D3, D), ix2(D, DD, 1),               // B = T1: k = (l1,u1), cols (r1,m)
                  ix2(Dc * Dc, D, D3), ix2(D, DD, 1));       // C = P2[a'][b][r1][l2][m]
    case 2:
      return gemm(Dc * Dc * D, DD, DD,
                  ix1(DD), kx(D, D, 1),                      // A = P2: rows (a',b,r1), k = (l2,m)
                  kx(D, D3, D), ix2(D, DD, 1),               // B = T2: k = (l2,m), cols (r2,d2)
                  ix2(Dc * D, D, D * Dc * D), ix2(D, Dc * D, 1));  // C = P3[b][r1][r2][a'][d2]
    default:
      return gemm(Dc * DD, Dc, Dc * D,
                  ix1(Dc * D), kx(D, D, 1),                  // A = P3: rows (b,r1,r2), k = (a',d2)
                  kx(D, D * Dc, Dc), ix1(1),                 // B = Md: k = (a',d2), cols b'
                  ix1(Dc), ix1(1));                          // C = E'[b][r1][r2][b']
  }
}

// Two-row right transfer:
//   H_c[a,l1,l2,a'] = sum Mu[a,u1,b] T1[l1,r1,u1,m] T2[l2,r2,m,d2] Md[a',d2,b'] H_{c+1}[b,r1,r2,b'].
//   s0: P1[a][r2][b'][u1][r1]  = Mu . H    (sum b)
//   s1: P2[a][r2][b'][l1][m]   = P1 . T1   (sum u1,r1)
//   s2: Q[a][l1][l2][d2][b']   = P2 . T2   (sum r2,m; batched over a)
//   s3: H'[a][l1][l2][a']      = Q . Md    (sum d2,b')
PEPS_HD GemmDesc col2_right_step(int s, int D, int Dc) {
  const int DD = D * D, D3 = D * D * D;
  switch (s) {
    case 0:
      return gemm(Dc * D, D * D * Dc, Dc,
                  ix1(Dc), kx(Dc, 0, 1),                     // A = Mu: rows (a,u1), k = b
                  kx(Dc, 0, DD * Dc), ix1(1),                // B = H[b][r1][r2][b']: cols (r1,r2,b')
                  ix2(D, Dc * D3, D), ix2(D * Dc, 1, DD));   // C = P1[a][r2][b'][u1][r1]
    case 1:
      return gemm(Dc * D * Dc, DD, DD,
                  ix1(DD), kx(D, D, 1),                      // A = P1: rows (a,r2,b'), k = (u1,r1)
                  kx(D, D, DD), ix2(D, D3, 1),               // B = T1: k = (u1,r1), cols (l1,m)
                  ix1(DD), ix1(1));                          // C = P2[a][r2][b'][l1][m]
    case 2: {
      // batched over a: rows (b',l1), k = (r2,m), cols (l2,d2)
      GemmDesc g = gemm(Dc * D, DD, DD,
                        ix2(D, DD, D), kx(D, Dc * DD, 1),    // A = P2 (per a)
                        kx(D, DD, D), ix2(D, D3, 1),         // B = T2: k = (r2,m), cols (l2,d2)
                        ix2(D, 1, DD * Dc), ix2(D, D * Dc, Dc));  // C = Q[a][l1][l2][d2][b']
      g.nb = Dc;
      g.sa = D * Dc * DD;
      g.sb = 0;
      g.sc = D3 * Dc;
      return g;
    }
    default:
      return gemm(Dc * DD, Dc, D * Dc,
                  ix1(D * Dc), kx(Dc, Dc, 1),                // A = Q: rows (a,l1,l2), k = (d2,b')
                  kx(Dc, Dc, 1), ix1(D * Dc),                // B = Md[a'][d2][b']: cols a'
                  ix1(Dc), ix1(1));                          // C = H'[a][l1][l2][a']
  }
}

// Number of steps and the buffer each step reads (A) / writes (C):
// buffer ids: 0 = input transfer, 1 = output transfer, 2.. = temporaries.
constexpr int kCol1Steps = 3, kSiteEnvSteps = 3, kCol2Steps = 4;

// ------------------------------------------------------------- zip-up steps
// Absorbing one row into a boundary MPS (Fig. 1d).  Actual (unpadded) bond
// dimensions are used: k = carry bond, a/b = old MPS bonds left/right of
// column c, i = physical index of the old MPS (= T's 'in' leg), l/r = T's
// horizontal legs, o = T's 'out' leg.  The site tensor is read padded with
// strides (sl, sr, si, so); MPS tensors are read padded [a][p][b].
struct ZipDims {
  int k, a, b, i, l, r, o;
};

// Left-to-right, column c:
//   s0: Y[k][b][l][i] = sum_a C[k][a][l] M[a][i][b]
//   s1: X[(k,o)][(b,r)] = sum_{l,i} Y[k][b][l][i] T[l][r][i][o]
PEPS_HD GemmDesc zip_lr_step(int s, const ZipDims& z, int D, int Dc, int sl, int sr, int si, int so) {
  if (s == 0)
    return gemm(z.k * z.l, z.i * z.b, z.a,
                ix2(z.l, z.a * z.l, 1), kx(z.a, 0, z.l),         // A = C[k][a][l]: rows (k,l)
                kx(z.a, 0, D * Dc), ix2(z.b, Dc, 1),             // B = M[a][i][b]: cols (i,b)
                ix2(z.l, z.b * z.l * z.i, z.i), ix2(z.b, 1, z.l * z.i));  // C = Y[k][b][l][i]
  return gemm(z.k * z.b, z.r * z.o, z.l * z.i,
              ix1(z.l * z.i), kx(z.i, z.i, 1),                   // A = Y: rows (k,b), k = (l,i)
              kx(z.i, sl, si), ix2(z.o, sr, so),                 // B = T: k = (l,i), cols (r,o)
              ix2(z.b, z.o * z.b * z.r, z.r), ix2(z.o, 1, z.b * z.r));  // C = X[(k,o)][(b,r)]
}

// Right-to-left, column c (carry C[b][r][k] comes from the right):
//   s0: Y[a][k][i][r] = sum_b M[a][i][b] C[b][r][k]
//   s1: X[(o,k)][(a,l)] = sum_{i,r} Y[a][k][i][r] T[l][r][i][o]
PEPS_HD GemmDesc zip_rl_step(int s, const ZipDims& z, int D, int Dc, int sl, int sr, int si, int so) {
  if (s == 0)
    return gemm(z.a * z.i, z.r * z.k, z.b,
                ix2(z.i, D * Dc, Dc), kx(z.b, 0, 1),             // A = M[a][i][b]: rows (a,i), k = b
                kx(z.b, 0, z.r * z.k), ix1(1),                   // B = C[b][r][k]: cols (r,k)
                ix2(z.i, z.k * z.i * z.r, z.r), ix2(z.k, 1, z.i * z.r));  // C = Y[a][k][i][r]
  return gemm(z.a * z.k, z.l * z.o, z.i * z.r,
              ix1(z.i * z.r), kx(z.r, z.r, 1),                   // A = Y: rows (a,k), k = (i,r)
              kx(z.r, si, sr), ix2(z.o, sl, so),                 // B = T: k = (i,r), cols (l,o)
              ix2(z.k, z.l, z.a * z.l), ix2(z.o, 1, z.k * z.a * z.l));  // C = X[(o,k)][(a,l)]
}

}  // namespace peps
