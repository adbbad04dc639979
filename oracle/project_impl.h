/*
 * Oracle projection of one splat (TEST INFRASTRUCTURE, see darb_oracle.c).
 *
 * This body is included twice by darb_oracle.c: once with REAL = float (the
 * fixed FP32 operation sequence whose results decide culling, radius, tile
 * rectangle, depth order and the per-pixel support test) and once with
 * REAL = double (the same formulas in FP64, used for finite-difference
 * checks).  Every rounded operation below is one IEEE operation; FMA() is a
 * fused multiply-add.  The file is compiled with -ffp-contract=off so that
 * the compiler adds no contraction of its own.
 *
 * Formulas (paper Sec. 4.1 "DARB Projection", Eq. 2x2covProjection, and the
 * correction-factor listings of supplementary Sec. B, "cov *= psi"):
 *   t      = W m + w                          (view transform)
 *   Sigma  = R(q) S S^T R(q)^T                (3DGS parameterisation, Sec. 4.1)
 *   J      = perspective Jacobian at t (guard band 1.3 tan(fov/2))
 *   Sigma' = J W Sigma W^T J^T, 2x2 block     (EWA, Sec. 4.1)
 *   Sigma2 = psi * Sigma' + 0.3 I             (psi of Table 2; low-pass dilation)
 *   conic  = Sigma2^-1, R = ceil(3 sqrt(lambda_max(Sigma2)))   (Sec. 4.1)
 */

static void PROJECT_FN(const float *mi, const float *si, const float *qi,
                       const orc_camera *cam, float psi_f, int tile, orc_proj *o)
{
    REAL V[16];
    for (int k = 0; k < 16; ++k) V[k] = (REAL)cam->viewmat[k];
    memset(o, 0, sizeof *o);
    o->culled = 1;

    /* view transform */
    REAL t[3];
    for (int r = 0; r < 3; ++r)
        t[r] = FMA(V[4 * r + 2], (REAL)mi[2],
                   FMA(V[4 * r + 1], (REAL)mi[1], FMA(V[4 * r + 0], (REAL)mi[0], V[4 * r + 3])));
    const REAL tz = t[2];
    if (!(tz > (REAL)cam->near_plane)) return; /* near-plane cull */

    /* unit quaternion (w, x, y, z) -> rotation */
    const REAL qw = qi[0], qx = qi[1], qy = qi[2], qz = qi[3];
    const REAL n2 = FMA(qz, qz, FMA(qy, qy, FMA(qx, qx, qw * qw)));
    if (!(n2 > (REAL)0) || !isfinite(n2)) return;
    const REAL inv = (REAL)1 / SQRT(n2);
    const REAL w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    const REAL xx = x * x, yy = y * y, zz = z * z;
    const REAL xy = x * y, xz = x * z, yz = y * z;
    const REAL wx = w * x, wy = w * y, wz = w * z;
    const REAL one = 1, two = 2;
    REAL R[3][3];
    R[0][0] = one - two * (yy + zz); R[0][1] = two * (xy - wz);       R[0][2] = two * (xz + wy);
    R[1][0] = two * (xy + wz);       R[1][1] = one - two * (xx + zz); R[1][2] = two * (yz - wx);
    R[2][0] = two * (xz - wy);       R[2][1] = two * (yz + wx);       R[2][2] = one - two * (xx + yy);

    /* Sigma = M M^T with M = R diag(s) */
    REAL M[3][3];
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) M[j][k] = R[j][k] * (REAL)si[k];
    REAL S[3][3];
    for (int j = 0; j < 3; ++j)
        for (int l = j; l < 3; ++l) {
            S[j][l] = FMA(M[j][2], M[l][2], FMA(M[j][1], M[l][1], M[j][0] * M[l][0]));
            S[l][j] = S[j][l];
        }

    /* perspective Jacobian with the guard band */
    const REAL fx = cam->fx, fy = cam->fy;
    const REAL txtz = t[0] / tz, tytz = t[1] / tz;
    const REAL limx = (REAL)1.3f * ((REAL)cam->width / (two * fx));
    const REAL limy = (REAL)1.3f * ((REAL)cam->height / (two * fy));
    o->clampx = (txtz < -limx) || (txtz > limx);
    o->clampy = (tytz < -limy) || (tytz > limy);
    const REAL txc = FMIN(limx, FMAX(-limx, txtz)) * tz;
    const REAL tyc = FMIN(limy, FMAX(-limy, tytz)) * tz;
    const REAL tz2 = tz * tz;
    const REAL J00 = fx / tz, J02 = -(fx * txc) / tz2;
    const REAL J11 = fy / tz, J12 = -(fy * tyc) / tz2;

    /* T = J W (2x3), Sigma' = T Sigma T^T (2x2) */
    REAL T0[3], T1[3], U0[3], U1[3];
    for (int k = 0; k < 3; ++k) {
        T0[k] = FMA(J02, V[8 + k], J00 * V[0 + k]);
        T1[k] = FMA(J12, V[8 + k], J11 * V[4 + k]);
    }
    for (int k = 0; k < 3; ++k) {
        U0[k] = FMA(T0[2], S[2][k], FMA(T0[1], S[1][k], T0[0] * S[0][k]));
        U1[k] = FMA(T1[2], S[2][k], FMA(T1[1], S[1][k], T1[0] * S[0][k]));
    }
    const REAL s00 = FMA(U0[2], T0[2], FMA(U0[1], T0[1], U0[0] * T0[0]));
    const REAL s01 = FMA(U0[2], T1[2], FMA(U0[1], T1[1], U0[0] * T1[0]));
    const REAL s11 = FMA(U1[2], T1[2], FMA(U1[1], T1[1], U1[0] * T1[0]));

    /* correction factor psi, then the 0.3 px^2 low-pass dilation */
    const REAL psi = psi_f;
    const REAL a = psi * s00 + (REAL)0.3f, b = psi * s01, c = psi * s11 + (REAL)0.3f;
    const REAL det = FMA(a, c, -(b * b));
    if (!(det > (REAL)0)) return;
    const REAL A = c / det, B = -b / det, C = a / det;

    /* larger eigenvalue and the 3-sigma radius */
    const REAL mid = (REAL)0.5f * (a + c);
    const REAL disc = FMA(mid, mid, -det);
    const REAL lam = mid + SQRT(FMAX(disc, (REAL)0));
    const REAL Rf = CEIL((REAL)3 * SQRT(lam));

    /* projected mean, pixel centres at integer + 0.5 */
    const REAL u0 = FMA(fx, txtz, (REAL)cam->cx), u1 = FMA(fy, tytz, (REAL)cam->cy);
    if (!isfinite(u0) || !isfinite(u1) || !isfinite(Rf)) return;

    /* pixel-exact rectangle of centres within [u - R, u + R], clamped to the image */
    const REAL half = (REAL)0.5f;
    const REAL x0 = FMAX(CEIL((u0 - Rf) - half), (REAL)0);
    const REAL x1 = FMIN(FLOOR((u0 + Rf) - half), (REAL)(cam->width - 1));
    const REAL y0 = FMAX(CEIL((u1 - Rf) - half), (REAL)0);
    const REAL y1 = FMIN(FLOOR((u1 + Rf) - half), (REAL)(cam->height - 1));
    if (!(x0 <= x1) || !(y0 <= y1)) return;
    const int ix0 = (int)x0, ix1 = (int)x1, iy0 = (int)y0, iy1 = (int)y1;
    o->rect[0] = ix0 / tile;
    o->rect[1] = iy0 / tile;
    o->rect[2] = ix1 / tile;
    o->rect[3] = iy1 / tile;
    o->tiles = (o->rect[2] - o->rect[0] + 1) * (o->rect[3] - o->rect[1] + 1);
    o->radius = (int)FMIN(Rf, (REAL)16777216);
    o->depth = (float)tz;
    o->mean2d[0] = (double)u0;
    o->mean2d[1] = (double)u1;
    o->conic[0] = (double)A;
    o->conic[1] = (double)B;
    o->conic[2] = (double)C;
    o->culled = 0;
}
