// jxf_adjoint.cuh -- hand-written reverse mode (vector-Jacobian products) of
// the single-phase, inviscid right-hand side of §3.2 (the differentiable
// solver of §6 with dt held fixed).
//
// R(U): W = prim(U) per cell; per face F = HLLC(recon(W-stencil));
// R_i = -sum_d (F_{i+1/2} - F_{i-1/2})/dx_d.  Given Rbar, the adjoint is
//   Fbar_f = (Rbar_f - Rbar_{f-1})/dx_d                  (transposed divergence)
//   (WLbar, WRbar) = HLLC^T Fbar, Sbar = recon^T (WLbar, WRbar) per face
//   Wbar_c = sum over the stencil slots that map to c    (atomic scatter)
//   Ubar_c = prim^T Wbar_c.
// Every branch (min/max of the wave speeds, sign(s*), the WENO weights'
// smooth dependence) is differentiated along the branch the forward pass
// takes.  Each face recomputes its forward intermediates.
#pragma once
#include "jxf_impl.cuh"

namespace jxf {

// --------------------------------------------------------------- WENO5 VJP --
// Reverse of one side of weno5_pair: value = centre + sum a_k e_k / sum a_k.
// Returns the adjoints of q_k and e_k (the centre's adjoint is vbar).  With
// omega the normalised weights, Delta = value - centre and
// g_k = vbar (e_k - Delta) / sum a (the adjoint of a_k):
//   Jiang-Shu, a_k = d_k/q_k^2:            qbar_k = -2 g_k a_k / q_k;
//   WENO5-Z, a_k = d_k (1 + tau/q_k), tau = |q_0 - q_2|:
//     qbar_k = -g_k d_k tau/q_k^2, taubar = sum_k g_k d_k/q_k,
//     qbar_0 += s taubar, qbar_2 -= s taubar with s = sign(q_0 - q_2)
//     (+1 at a tie, the branch the forward takes).
template <typename T>
__device__ __forceinline__ void weno5_side_vjp(T q0, T q1, T q2, T e0, T e1, T e2, T vbar, bool z,
                                               T &qb0, T &qb1, T &qb2, T &eb0, T &eb1, T &eb2) {
    const T r0 = rcp(q0), r1 = rcp(q1), r2 = rcp(q2);
    if (z) {
        const T dq = q0 - q2;
        const T tau = dq < T(0) ? -dq : dq;
        const T s = dq < T(0) ? T(-1) : T(1);
        const T w0 = T(0.1) * (T(1) + tau * r0), w1 = T(0.6) * (T(1) + tau * r1);
        const T w2 = T(0.3) * (T(1) + tau * r2);
        const T iw = rcp(w0 + w1 + w2);
        const T o0 = w0 * iw, o1 = w1 * iw, o2 = w2 * iw;
        const T delta = o0 * e0 + o1 * e1 + o2 * e2;
        eb0 = vbar * o0;
        eb1 = vbar * o1;
        eb2 = vbar * o2;
        const T g0 = vbar * (e0 - delta) * iw, g1 = vbar * (e1 - delta) * iw;
        const T g2 = vbar * (e2 - delta) * iw;
        qb0 = -g0 * T(0.1) * tau * r0 * r0;
        qb1 = -g1 * T(0.6) * tau * r1 * r1;
        qb2 = -g2 * T(0.3) * tau * r2 * r2;
        const T taub = g0 * T(0.1) * r0 + g1 * T(0.6) * r1 + g2 * T(0.3) * r2;
        qb0 += s * taub;
        qb2 -= s * taub;
        return;
    }
    const T w0 = T(0.1) * r0 * r0, w1 = T(0.6) * r1 * r1, w2 = T(0.3) * r2 * r2;
    const T iw = rcp(w0 + w1 + w2);
    const T o0 = w0 * iw, o1 = w1 * iw, o2 = w2 * iw;
    const T delta = o0 * e0 + o1 * e1 + o2 * e2;
    eb0 = vbar * o0;
    eb1 = vbar * o1;
    eb2 = vbar * o2;
    qb0 = vbar * T(-2) * o0 * (e0 - delta) * r0;
    qb1 = vbar * T(-2) * o1 * (e1 - delta) * r1;
    qb2 = vbar * T(-2) * o2 * (e2 - delta) * r2;
}

// Reverse of weno5_pair: accumulates into xb[0..5] the adjoint of the six
// cell values given the adjoints of the left and right face values.
template <typename T>
__device__ __forceinline__ void weno5_pair_vjp(const T (&x)[6], T eps, bool z, T vlb, T vrb,
                                               T (&xb)[6]) {
    const T D0 = x[1] - x[0], D1 = x[2] - x[1], D2 = x[3] - x[2];
    const T D3 = x[4] - x[3], D4 = x[5] - x[4];
    const T k13 = T(1.0408329997330663);
    const T a0 = (D1 - D0) * k13, a1 = (D2 - D1) * k13;
    const T a2 = (D3 - D2) * k13, a3 = (D4 - D3) * k13;
    const T c0 = a0 * a0 + eps, c1 = a1 * a1 + eps, c2 = a2 * a2 + eps, c3 = a3 * a3 + eps;
    const T sixth = T(1.0 / 6.0);
    T Db0 = 0, Db1 = 0, Db2 = 0, Db3 = 0, Db4 = 0;
    T ab0 = 0, ab1 = 0, ab2 = 0, ab3 = 0;
    {  // left
        const T h0 = T(1.5) * D1 - T(0.5) * D0, h1 = T(0.5) * (D1 + D2), h2 = T(0.5) * D3 - T(1.5) * D2;
        const T q0 = h0 * h0 + c0, q1 = h1 * h1 + c1, q2 = h2 * h2 + c2;
        const T e0 = (T(5) * D1 - T(2) * D0) * sixth, e1 = (D1 + T(2) * D2) * sixth;
        const T e2 = (T(4) * D2 - D3) * sixth;
        T qb0, qb1, qb2, eb0, eb1, eb2;
        weno5_side_vjp(q0, q1, q2, e0, e1, e2, vlb, z, qb0, qb1, qb2, eb0, eb1, eb2);
        xb[2] += vlb;
        // e
        Db1 += (T(5) * eb0 + eb1) * sixth;
        Db0 += T(-2) * eb0 * sixth;
        Db2 += (T(2) * eb1 + T(4) * eb2) * sixth;
        Db3 += -eb2 * sixth;
        // q = h^2 + a^2 + eps
        const T hb0 = T(2) * h0 * qb0, hb1 = T(2) * h1 * qb1, hb2 = T(2) * h2 * qb2;
        ab0 += T(2) * a0 * qb0;
        ab1 += T(2) * a1 * qb1;
        ab2 += T(2) * a2 * qb2;
        Db1 += T(1.5) * hb0 + T(0.5) * hb1;
        Db0 += T(-0.5) * hb0;
        Db2 += T(0.5) * hb1 - T(1.5) * hb2;
        Db3 += T(0.5) * hb2;
    }
    {  // right (mirrored)
        const T h0 = T(0.5) * D4 - T(1.5) * D3, h1 = T(0.5) * (D2 + D3), h2 = T(1.5) * D2 - T(0.5) * D1;
        const T q0 = h0 * h0 + c3, q1 = h1 * h1 + c2, q2 = h2 * h2 + c1;
        const T e0 = (T(2) * D4 - T(5) * D3) * sixth, e1 = -(D3 + T(2) * D2) * sixth;
        const T e2 = (D1 - T(4) * D2) * sixth;
        T qb0, qb1, qb2, eb0, eb1, eb2;
        weno5_side_vjp(q0, q1, q2, e0, e1, e2, vrb, z, qb0, qb1, qb2, eb0, eb1, eb2);
        xb[3] += vrb;
        Db4 += T(2) * eb0 * sixth;
        Db3 += (T(-5) * eb0 - eb1) * sixth;
        Db2 += (T(-2) * eb1 - T(4) * eb2) * sixth;
        Db1 += eb2 * sixth;
        const T hb0 = T(2) * h0 * qb0, hb1 = T(2) * h1 * qb1, hb2 = T(2) * h2 * qb2;
        ab3 += T(2) * a3 * qb0;
        ab2 += T(2) * a2 * qb1;
        ab1 += T(2) * a1 * qb2;
        Db4 += T(0.5) * hb0;
        Db3 += T(-1.5) * hb0 + T(0.5) * hb1;
        Db2 += T(0.5) * hb1 + T(1.5) * hb2;
        Db1 += T(-0.5) * hb2;
    }
    // a_k = k13 (D_{k+1} - D_k)
    Db1 += k13 * ab0;
    Db0 -= k13 * ab0;
    Db2 += k13 * ab1;
    Db1 -= k13 * ab1;
    Db3 += k13 * ab2;
    Db2 -= k13 * ab2;
    Db4 += k13 * ab3;
    Db3 -= k13 * ab3;
    // D_k = x_{k+1} - x_k
    xb[1] += Db0;
    xb[0] -= Db0;
    xb[2] += Db1;
    xb[1] -= Db1;
    xb[3] += Db2;
    xb[2] -= Db2;
    xb[4] += Db3;
    xb[3] -= Db3;
    xb[5] += Db4;
    xb[4] -= Db4;
}

// ----------------------------------------------------- reconstruction VJP --
// Reverse of reconstruct() for the single-phase model: Sb[j][v] accumulates
// the adjoint of the six stencil primitives from the face-state adjoints.
template <typename T, int NDIM, int d>
__device__ __forceinline__ void reconstruct_vjp(const Dev &P, const T (&S)[6][MAXV], const T *WLb,
                                                const T *WRb, T (&Sb)[6][MAXV]) {
    using V = Vars<JXF_SPM, NDIM>;
    constexpr int NV = V::NV, IE = V::IE, in = 1 + d;
    const T eps = cst<T>(P).weno_eps;
    const bool z = P.weno_z != 0;
    if (P.recon == JXF_WENO5JS_COMP) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T x[6] = {S[0][v], S[1][v], S[2][v], S[3][v], S[4][v], S[5][v]};
            T xb[6] = {0, 0, 0, 0, 0, 0};
            weno5_pair_vjp(x, eps, z, WLb[v], WRb[v], xb);
#pragma unroll
            for (int j = 0; j < 6; ++j) Sb[j][v] += xb[j];
        }
        return;
    }
    // forward: frozen state and projection
    const Cst<T> &C = cst<T>(P);
    T Wb[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Wb[v] = T(0.5) * (S[2][v] + S[3][v]);
    const T rho = Wb[0];
    const T rc2 = C.gamma0 * (Wb[IE] + C.pinf0);
    const T irc2 = rcp(rc2);
    const T irho = rcp(rho);
    const T xcs = rc2 * irho;
    const T cb = dsqrt(xcs);
    const T icb = rcp(cb);
    const T h_c = T(0.5) * icb;
    const T h_rc2 = T(0.5) * irc2;
    const T ent = Wb[0] * irc2;
    T q[MAXV][6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
        for (int v = 0; v < NV; ++v) q[v][j] = S[j][v];
        q[0][j] = S[j][0] - ent * S[j][IE];
        q[in][j] = -h_c * S[j][in] + h_rc2 * S[j][IE];
        q[IE][j] = h_c * S[j][in] + h_rc2 * S[j][IE];
    }
    T qL[MAXV], qR[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (z) weno5_pair<true>(q[v], cst<T>(P).weno_eps4, qL[v], qR[v]);
        else weno5_pair<false>(q[v], cst<T>(P).weno_eps4, qL[v], qR[v]);
    }
    // reverse of the back-projection o = K q (both sides)
    T qLb[MAXV], qRb[MAXV];
    T Wb0b = 0, cbb = 0, rc2b = 0;
    const T *ob[2] = {WLb, WRb};
    const T *qs[2] = {qL, qR};
    T *qbs[2] = {qLb, qRb};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const T *o = ob[s];
        const T *qq = qs[s];
        T *qb = qbs[s];
#pragma unroll
        for (int v = 0; v < NV; ++v) qb[v] = o[v];
        // o[0] = Wb0 q[in] + q[0] + Wb0 q[IE]
        qb[0] = o[0];
        qb[in] = o[0] * Wb[0];
        qb[IE] = o[0] * Wb[0];
        Wb0b += o[0] * (qq[in] + qq[IE]);
        // o[in] = cb (q[IE] - q[in])
        qb[IE] += o[in] * cb;
        qb[in] -= o[in] * cb;
        cbb += o[in] * (qq[IE] - qq[in]);
        // o[IE] = rc2 (q[in] + q[IE])
        qb[in] += o[IE] * rc2;
        qb[IE] += o[IE] * rc2;
        rc2b += o[IE] * (qq[in] + qq[IE]);
    }
    // reverse of the WENO reconstructions
    T qb[MAXV][6];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
        for (int j = 0; j < 6; ++j) qb[v][j] = T(0);
        weno5_pair_vjp(q[v], eps, z, qLb[v], qRb[v], qb[v]);
    }
    // reverse of the projection q = K^{-1} S
    T entb = 0, h_cb = 0, h_rc2b = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if (v != 0 && v != in && v != IE) Sb[j][v] += qb[v][j];
        // q0 = S0 - ent S_IE
        Sb[j][0] += qb[0][j];
        Sb[j][IE] -= qb[0][j] * ent;
        entb -= qb[0][j] * S[j][IE];
        // q_in = -h_c S_in + h_rc2 S_IE ; q_IE = h_c S_in + h_rc2 S_IE
        Sb[j][in] += (qb[IE][j] - qb[in][j]) * h_c;
        Sb[j][IE] += (qb[IE][j] + qb[in][j]) * h_rc2;
        h_cb += (qb[IE][j] - qb[in][j]) * S[j][in];
        h_rc2b += (qb[IE][j] + qb[in][j]) * S[j][IE];
    }
    // frozen-state intermediates
    T irc2b = entb * Wb[0] + T(0.5) * h_rc2b;
    Wb0b += entb * irc2;
    cbb -= h_cb * h_c * icb;
    const T xb = cbb * (T(0.5) * icb);
    rc2b += xb * irho;
    Wb0b -= xb * xcs * irho;  // rho = Wb[0]
    rc2b -= irc2b * irc2 * irc2;
    T Wbb[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Wbb[v] = T(0);
    Wbb[0] = Wb0b;
    Wbb[IE] += rc2b * C.gamma0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        Sb[2][v] += T(0.5) * Wbb[v];
        Sb[3][v] += T(0.5) * Wbb[v];
    }
}

// ---------------------------------------------------------------- HLLC VJP --
// Reverse of hllc() for the single-phase model: from the adjoint of the face
// flux (Fb, uhb ignored: inviscid single phase has no face-velocity source)
// to the adjoints of the two primitive face states.
template <typename T, int NDIM, int d>
__device__ __forceinline__ void hllc_vjp(const Dev &P, const T *WL, const T *WR, const T *Fb,
                                         T *WLb, T *WRb) {
    using V = Vars<JXF_SPM, NDIM>;
    constexpr int NV = V::NV, IE = V::IE, in = 1 + d;
    const Cst<T> &C = cst<T>(P);
    const T g = C.gamma0, pinf = C.pinf0, A = C.A1;  // A = 1/(gamma-1)
    // ---- forward
    const T rhoL = WL[0], rhoR = WR[0], uL = WL[in], uR = WR[in], pL = WL[IE], pR = WR[IE];
    const T irhoL = rcp(rhoL), irhoR = rcp(rhoR);
    const T c2L = g * (pL + pinf) * irhoL, c2R = g * (pR + pinf) * irhoR;
    const T cL = dsqrt(c2L), cR = dsqrt(c2R);
    const T srL = dsqrt(rhoL), srR = dsqrt(rhoR);
    const T is = rcp(srL + srR);
    const T S2 = srL * uL + srR * uR;
    const T ubar = S2 * is;
    const T du = uR - uL;
    const T S1 = srL * c2L + srR * c2R;
    const T c2bar = S1 * is + T(0.5) * srL * srR * is * is * du * du;
    const T cbar = dsqrt(c2bar);
    const bool Lfirst = !((uL - cL) < (ubar - cbar));  // tmin picks uL-cL when smaller
    const T sL = Lfirst ? ubar - cbar : uL - cL;
    const bool Rfirst = !((uR + cR) > (ubar + cbar));
    const T sR = Rfirst ? ubar + cbar : uR + cR;
    const T mL = rhoL * (sL - uL), mR = rhoR * (sR - uR);
    const T num = pR - pL + mL * uL - mR * uR, den2 = mL - mR;
    const T iden2 = rcp(den2);
    const T sstar = num * iden2;
    const T sm = sL < T(0) ? sL : T(0), sp = sR > T(0) ? sR : T(0);
    const int first = sstar < T(0) ? 1 : 0, last = sstar > T(0) ? 0 : 1;
    const T wgt = first == last ? T(1) : T(0.5);
    // ---- reverse
    T sLb = 0, sRb = 0, smb = 0, spb = 0, ssb = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        WLb[v] = T(0);
        WRb[v] = T(0);
    }
#pragma unroll 1
    for (int side = first; side <= last; ++side) {
        const bool R = side == 1;
        T W[MAXV], Wbk[MAXV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            W[v] = R ? WR[v] : WL[v];
            Wbk[v] = T(0);
        }
        const T sK = R ? sR : sL, sPM = R ? sp : sm;
        const T rho = W[0], u = W[in], p = W[IE];
        T uu = T(0);
#pragma unroll
        for (int e = 0; e < NDIM; ++e) uu += W[1 + e] * W[1 + e];
        const T E = (p + C.gpinf0) * A + T(0.5) * rho * uu;
        T U[MAXV];
        U[0] = rho;
#pragma unroll
        for (int e = 0; e < NDIM; ++e) U[1 + e] = rho * W[1 + e];
        U[IE] = E;
        const T su = sK - u, den = sK - sstar;
        const T isu = rcp(su), iden = rcp(den);
        const T fac = su * iden;
        const T B = rho * sstar + p * isu;
        const T Aterm = E + (sstar - u) * B;
        T Us[MAXV];
        Us[0] = fac * rho;
#pragma unroll
        for (int e = 0; e < NDIM; ++e) Us[1 + e] = fac * (rho * W[1 + e]);
        Us[in] = fac * (rho * sstar);
        Us[IE] = fac * Aterm;
        // F = wgt (Fp + sPM (Us - U));  Fp: mass rho u, momentum U_e u (+p), energy u (E+p)
        T Fpb[MAXV], Usb[MAXV], Ub[MAXV];
        T sPMb = T(0);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T fb = wgt * Fb[v];
            Fpb[v] = fb;
            Usb[v] = sPM * fb;
            Ub[v] = -sPM * fb;
            sPMb += fb * (Us[v] - U[v]);
        }
        T ub = T(0), pb = T(0), rhob = T(0), Eb = T(0), facb = T(0), ssk = T(0);
        // physical flux
        Ub[0] += Fpb[0] * u;
        ub += Fpb[0] * U[0];
#pragma unroll
        for (int e = 0; e < NDIM; ++e) {
            Ub[1 + e] += Fpb[1 + e] * u;
            ub += Fpb[1 + e] * U[1 + e];
        }
        pb += Fpb[in];
        ub += Fpb[IE] * (E + p);
        Eb += Fpb[IE] * u;
        pb += Fpb[IE] * u;
        // star state
        facb += Usb[0] * rho;
        rhob += Usb[0] * fac;
#pragma unroll
        for (int e = 0; e < NDIM; ++e) {
            if (e == d) continue;
            facb += Usb[1 + e] * rho * W[1 + e];
            rhob += Usb[1 + e] * fac * W[1 + e];
            Wbk[1 + e] += Usb[1 + e] * fac * rho;
        }
        facb += Usb[in] * rho * sstar;
        rhob += Usb[in] * fac * sstar;
        ssk += Usb[in] * fac * rho;
        facb += Usb[IE] * Aterm;
        const T Ab = Usb[IE] * fac;
        Eb += Ab;
        ssk += Ab * B;
        ub -= Ab * B;
        const T Bb = Ab * (sstar - u);
        rhob += Bb * sstar;
        ssk += Bb * rho;
        pb += Bb * isu;
        T sub = -Bb * p * (isu * isu);
        // fac = su / den
        sub += facb * iden;
        const T denb = -facb * fac * iden;
        T sKb = denb + sub;
        ssk -= denb;
        ub -= sub;
        // U = prim2cons(W)
        rhob += Ub[0];
#pragma unroll
        for (int e = 0; e < NDIM; ++e) {
            rhob += Ub[1 + e] * W[1 + e];
            Wbk[1 + e] += Ub[1 + e] * rho;
        }
        Eb += Ub[IE];
        rhob += Eb * T(0.5) * uu;
#pragma unroll
        for (int e = 0; e < NDIM; ++e) Wbk[1 + e] += Eb * rho * W[1 + e];
        pb += Eb * A;
        Wbk[0] += rhob;
        Wbk[in] += ub;
        Wbk[IE] += pb;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            if (R) WRb[v] += Wbk[v];
            else WLb[v] += Wbk[v];
        }
        if (R) {
            sRb += sKb;
            spb += sPMb;
        } else {
            sLb += sKb;
            smb += sPMb;
        }
        ssb += ssk;
    }
    // sm = min(0, sL), sp = max(0, sR)
    if (sL < T(0)) sLb += smb;
    if (sR > T(0)) sRb += spb;
    // s* = num / den2
    const T numb = ssb * iden2;
    const T den2b = -ssb * sstar * iden2;
    T mLb = numb * uL + den2b, mRb = -numb * uR - den2b;
    T pLb = -numb, pRb = numb, uLb = numb * mL, uRb = -numb * mR, rhoLb = 0, rhoRb = 0;
    // m = rho (s - u)
    rhoLb += mLb * (sL - uL);
    sLb += mLb * rhoL;
    uLb -= mLb * rhoL;
    rhoRb += mRb * (sR - uR);
    sRb += mRb * rhoR;
    uRb -= mRb * rhoR;
    // wave speeds
    T ubarb = 0, cbarb = 0, cLb = 0, cRb = 0;
    if (Lfirst) {
        ubarb += sLb;
        cbarb -= sLb;
    } else {
        uLb += sLb;
        cLb -= sLb;
    }
    if (Rfirst) {
        ubarb += sRb;
        cbarb += sRb;
    } else {
        uRb += sRb;
        cRb += sRb;
    }
    const T c2barb = cbarb * (T(0.5) * rcp(cbar));
    // c2bar = S1 is + 0.5 srL srR is^2 du^2
    const T S1b = c2barb * is;
    T isb = c2barb * S1 + c2barb * srL * srR * is * du * du;
    T srLb = c2barb * T(0.5) * srR * is * is * du * du;
    T srRb = c2barb * T(0.5) * srL * is * is * du * du;
    const T dub = c2barb * srL * srR * is * is * du;
    uRb += dub;
    uLb -= dub;
    T c2Lb = S1b * srL, c2Rb = S1b * srR;
    srLb += S1b * c2L;
    srRb += S1b * c2R;
    // ubar = S2 is
    const T S2b = ubarb * is;
    isb += ubarb * S2;
    srLb += S2b * uL;
    uLb += S2b * srL;
    srRb += S2b * uR;
    uRb += S2b * srR;
    // is = 1/(srL + srR)
    const T sumb = -isb * is * is;
    srLb += sumb;
    srRb += sumb;
    rhoLb += srLb * (T(0.5) * rcp(srL));
    rhoRb += srRb * (T(0.5) * rcp(srR));
    c2Lb += cLb * (T(0.5) * rcp(cL));
    c2Rb += cRb * (T(0.5) * rcp(cR));
    // c2 = g (p + pinf) / rho
    pLb += c2Lb * g * irhoL;
    rhoLb -= c2Lb * c2L * irhoL;
    pRb += c2Rb * g * irhoR;
    rhoRb -= c2Rb * c2R * irhoR;
    WLb[0] += rhoLb;
    WLb[in] += uLb;
    WLb[IE] += pLb;
    WRb[0] += rhoRb;
    WRb[in] += uRb;
    WRb[IE] += pRb;
}

// Start of axis d's section of the stencil-slot adjoints: the axes' sections
// ([slot][variable][face] each) follow one another.
__host__ __device__ inline size_t sbar_offset(const Dev &P, int ndim, int d, int nv) {
    size_t off = 0;
    for (int e = 0; e < d && e < ndim; ++e) {
        size_t nf = 1;
        for (int k = 0; k < 3; ++k) nf *= (size_t)(P.n[k] + (k == e ? 1 : 0));
        off += 6 * (size_t)nv * nf;
    }
    return off;
}

// ----------------------------------------------------------- k_flux_vjp ----
// One thread per face of axis d: Fbar from Rbar (transposed divergence),
// forward recomputation, reverse through HLLC and the reconstruction; the
// adjoints of the six stencil cells go to the face's slots of P.Sbar
// ([slot j][variable][face], mirrored slots with the normal velocity flipped
// back), and k_gather_vjp adds them to Wbar cell by cell in a fixed order --
// no atomics, so reverse mode gives the same bits on every run.
template <typename T, int NDIM, int d>
__global__ void __launch_bounds__(kFluxThreads) k_flux_vjp(const Dev P) {
    using V = Vars<JXF_SPM, NDIM>;
    constexpr int NV = V::NV;
    int m[3] = {P.n[0], P.n[1], P.n[2]};
    m[d] += 1;
    const long long nface = (long long)m[0] * m[1] * m[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nface) return;
    const unsigned gu = (unsigned)g;
    const unsigned q0 = P.fd_face[d][0].div(gu);
    const unsigned q1 = P.fd_face[d][1].div(q0);
    int c[3] = {(int)(gu - q0 * (unsigned)m[0]), (int)(q0 - q1 * (unsigned)m[1]), (int)q1};
    const int sd = d == 0 ? 1 : (d == 1 ? P.n[0] : P.n[0] * P.n[1]);
    const int base = ((c[2] * P.n[1] + c[1]) * P.n[0] + c[0]) - c[d] * sd;
    const size_t nc = (size_t)P.ncell;
    // Fbar_f = (Rbar_f - Rbar_{f-1}) / dx_d, cells outside the line contribute 0
    const T *Rb = static_cast<const T *>(P.Rbar);
    const T idx_d = cst<T>(P).inv_dx[d];
    T Fb[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const T right = c[d] < P.n[d] ? Rb[v * nc + chk_cell(P, base + c[d] * sd)] : T(0);
        const T left = c[d] > 0 ? Rb[v * nc + chk_cell(P, base + (c[d] - 1) * sd)] : T(0);
        Fb[v] = (right - left) * idx_d;
    }
    int idx[6];
    unsigned mir = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        int mj = 0;
        const int cj = map_axis(c[d] + j - 3, P.n[d], P.bc[d][0], P.bc[d][1], mj, 1);
        idx[j] = chk_cell(P, base + cj * sd);
        mir |= (unsigned)mj << j;
    }
    const T *W = static_cast<const T *>(P.W);
    T S[6][MAXV];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
        for (int v = 0; v < NV; ++v) S[j][v] = __ldg(W + v * nc + idx[j]);
        if ((mir >> j) & 1u) S[j][1 + d] = -S[j][1 + d];
    }
    T WL[MAXV], WR[MAXV];
    reconstruct<T, JXF_SPM, NDIM, d, 0>(P, S, WL, WR);  // WENO5: no reverse mode for TENO6-A
    T WLb[MAXV], WRb[MAXV];
    hllc_vjp<T, NDIM, d>(P, WL, WR, Fb, WLb, WRb);
    T Sb[6][MAXV];
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
        for (int v = 0; v < NV; ++v) Sb[j][v] = T(0);
    reconstruct_vjp<T, NDIM, d>(P, S, WLb, WRb, Sb);
    T *Sbar = static_cast<T *>(P.Sbar) + sbar_offset(P, NDIM, d, NV);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        if ((mir >> j) & 1u) Sb[j][1 + d] = -Sb[j][1 + d];
#pragma unroll
        for (int v = 0; v < NV; ++v) Sbar[((size_t)j * NV + v) * (size_t)nface + (size_t)g] = Sb[j][v];
    }
}

// Wbar of every cell = the sum of the stencil-slot adjoints of the faces
// whose stencils reach it, axis by axis (one thread per cell, after every axis's k_flux_vjp).
// Face f (between cells f-1 and f) holds slot j = cell f-3+j mapped through
// the boundary conditions; away from the ends of the line that is cell
// f-3+j itself, so cell i collects slot j of face i+3-j for j = 0..5; within
// three cells of an end every face near either end and near the cell is
// tested against the map.  The order of the additions is fixed, so the
// result is reproducible.
template <typename T, int NDIM, int d>
__device__ __forceinline__ void gather_axis(const Dev &P, const int (&c)[3], T *acc) {
    constexpr int NV = Vars<JXF_SPM, NDIM>::NV;
    int m[3] = {P.n[0], P.n[1], P.n[2]};
    m[d] += 1;
    const size_t nface = (size_t)m[0] * m[1] * m[2];
    const int n = P.n[d], ci = c[d];
    const int fs = d == 0 ? 1 : (d == 1 ? m[0] : m[0] * m[1]);  // face stride along d
    const int f0 = (c[2] * m[1] + c[1]) * m[0] + c[0] - ci * fs;  // face 0 of the cell's line
    const T *Sbar = static_cast<const T *>(P.Sbar) + sbar_offset(P, NDIM, d, NV);
    // slots hold the adjoint of the mapped cell (mirror flips already applied)
    auto take = [&](int f, int j) {
#pragma unroll
        const int g = chk_face(P, (long long)f0 + (long long)f * fs, (long long)nface);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += Sbar[((size_t)j * NV + v) * nface + (size_t)g];
    };
    if (ci >= 3 && ci <= n - 4) {
#pragma unroll
        for (int j = 0; j < 6; ++j) take(ci + 3 - j, j);
        return;
    }
    // faces within 7 of either end, then those within 3 of the cell
    const int e1 = min(n, 7), s2 = max(e1 + 1, n - 7);
    for (int part = 0; part < 3; ++part) {
        const int lo = part == 0 ? 0 : (part == 1 ? s2 : max(0, ci - 2));
        const int hi = part == 0 ? e1 : (part == 1 ? n : min(n, ci + 3));
        for (int f = lo; f <= hi; ++f) {
            if (part == 2 && (f <= e1 || f >= s2)) continue;
            for (int j = 0; j < 6; ++j) {
                int mj = 0;
                if (map_axis(f + j - 3, n, P.bc[d][0], P.bc[d][1], mj, 1) == ci) take(f, j);
            }
        }
    }
}

template <typename T, int NDIM>
__global__ void __launch_bounds__(kCellThreads) k_gather_vjp(const Dev P) {
    constexpr int NV = Vars<JXF_SPM, NDIM>::NV;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.ncell) return;
    const unsigned iu = (unsigned)i;
    const unsigned qy = P.fd_cell[0].div(iu), qz = P.fd_cell[1].div(qy);
    const int c[3] = {(int)(iu - qy * (unsigned)P.n[0]), (int)(qy - qz * (unsigned)P.n[1]), (int)qz};
    T *Wb = static_cast<T *>(P.Wbar);  // written here only: no clearing needed
    const size_t nc = (size_t)P.ncell;
    T w[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = T(0);
    gather_axis<T, NDIM, 0>(P, c, w);
    if constexpr (NDIM > 1) gather_axis<T, NDIM, 1>(P, c, w);
    if constexpr (NDIM > 2) gather_axis<T, NDIM, 2>(P, c, w);
#pragma unroll
    for (int v = 0; v < NV; ++v) Wb[v * nc + (size_t)i] = w[v];
}

// Ubar = (dW/dU)^T Wbar per cell (§2.1 state vectors, ideal / stiffened gas).
template <typename T, int NDIM>
__global__ void __launch_bounds__(kCellThreads) k_prim_vjp(const Dev P) {
    using V = Vars<JXF_SPM, NDIM>;
    constexpr int NV = V::NV, IE = V::IE;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.ncell) return;
    const T *U = static_cast<const T *>(P.Us);
    const T *Wb = static_cast<const T *>(P.Wbar);
    T *Ub = static_cast<T *>(P.Ubar);
    const T gm1 = cst<T>(P).gm1_0;
    const T rho = U[i];
    const T ir = rcp(rho);
    T u[3], wb[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) wb[v] = Wb[v * P.ncell + i];
    T uu = T(0);
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        u[e] = U[(1 + e) * P.ncell + i] * ir;
        uu += u[e] * u[e];
    }
    // p = (gamma-1)(E - 1/2 sum m_e u_e) - gamma pinf
    T rb = wb[0] + wb[IE] * gm1 * T(0.5) * uu;
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        rb -= wb[1 + e] * u[e] * ir;
        Ub[(1 + e) * P.ncell + i] = wb[1 + e] * ir - wb[IE] * gm1 * u[e];
    }
    Ub[i] = rb;
    Ub[IE * P.ncell + i] = wb[IE] * gm1;
}

// out = a x + b y + c z (elementwise over n values; y, z may be null).
template <typename T>
__global__ void k_axpbypcz(T *out, long long n, double a, const T *x, double b, const T *y, double c,
                           const T *z) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    T s = T(a) * x[k];
    if (y) s += T(b) * y[k];
    if (z) s += T(c) * z[k];
    out[k] = s;
}

}  // namespace jxf
