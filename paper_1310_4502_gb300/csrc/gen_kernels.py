#!/usr/bin/env python3
"""Generate the straight-line multipole routines of the CUDA library.

The paper produces its high-order interaction routines by metaprogramming
(computer-algebra output translated into C, Sec. "Multipole Error Bounds"); this
script plays that role for the GPU path.  It writes ``generated.cuh`` with, for
every order p = 0..6:

* ``m2p_eval<P>(rec, rx, ry, rz, phi, ax, ay, az)`` (P <= PMAX) -- one cell-to-particle
  interaction of the Cartesian expansion of the softened kernel
  F(R) = (|R|^2 + eps^2)^{-1/2}, written in a traced form:
      Phi(R) = sum_a (-1)^|a| / a!  d^a F(R) M_a
             = rho * sum_{k} w^k sum_{|b| <= p-2k} C_{b,k} y^b,
  with u = |R|^2 + eps^2, rho = u^{-1/2}, w = 1/u, y = R w, and per-cell
  coefficients
      C_{b,k} = (-1)^k (2m-1)!! / (2^k b!) * sum_{|l|=k} M_{b+2l} / l!,  m = |b|+k.
  The gradient follows from d rho/dR = -rho y, dw/dR = -2 w y,
  dy_e/dR_d = w delta_ed - 2 y_e y_d:
      dPhi/dR_d = rho [ w sum_k w^k dS_k/dy_d - y_d sum_{k,n} w^k (1+2k+2n) S_{k,n} ],
  S_{k,n} being the degree-n part of S_k.  The potential is -G Phi and the
  acceleration +G grad Phi.
* ``m2p_record<P>(M, inv_s, G, eps, rec)`` -- raw moments (FP64) to the record
  read by ``m2p_eval``: every coefficient is scaled by a power of two
  s = 1/inv_s (exact), so that R' = R/s and the coefficients stay O(1) in
  single precision; G/s is folded in.  Layout: [inv_s, eps^2/s^2, centre hi (3),
  centre lo (3), C_{b,k} ... in the order the evaluation reads them].  The gradient
  polynomials dS_k/dy_d are not stored: the evaluation forms them from the C_{b,k}
  by derivative-carrying Horner chains.
* the moment-translation (M2M) pair tables and multi-index tables.

``M2P_FLOPS[P]`` is a fixed roofline convention: the operation count (FMA = 2, the
rsqrt as 1) of the first, explicit-monomial form of this routine.  The shipped Horner
form does the same mathematics in fewer operations; ``m2p_source_flops(P)`` counts the
arithmetic operators of the shipped statements (FMA = 2, rsqrt = 1), so both figures
can be reported side by side.

Run: python gen_kernels.py  (rewrites generated.cuh next to this file).
"""
import math
import os
import sys

PMAX = 8      # largest expansion order of the forces
ADJ_PMAX = 6  # largest order of the adjoint's routines and tables
HDR = 8  # record header slots: inv_s, eps^2/s^2, centre hi (3), centre lo (3)


def midx(p):
    out = []
    for n in range(p + 1):
        for i in range(n, -1, -1):
            for j in range(n - i, -1, -1):
                out.append((i, j, n - i - j))
    return out


def ncomp(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def fact3(a):
    return math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2])


def add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def mname(a):
    return f"y{a[0]}{a[1]}{a[2]}"


def s_terms(p):
    """(k, n, beta) triples of the traced coefficients, in record order."""
    out = []
    for k in range(p // 2 + 1):
        for n in range(p - 2 * k + 1):
            for b in midx(n)[ncomp(n - 1) if n > 0 else 0:]:
                out.append((k, n, b))
    return out


# Flops per M2P interaction used as the roofline convention (FMA = 2, rsqrt = 1): the
# operation count of the traced expansion evaluated with explicit monomials (the first
# form of this routine, p = 0..8).  The Horner form below does the same mathematics with
# fewer instructions; the convention stays fixed so that rates stay comparable.
M2P_FLOP_CONVENTION = [32, 40, 82, 164, 307, 534, 874, 1358, 2023]


def _count_ops(stmt):
    """Arithmetic operations of one generated statement: every binary +, -, * and every
    compound assignment counts 1 (so a multiply-add counts 2), hot_rsqrt counts 1; unary
    minus and the coefficient references do not count."""
    import re
    t = re.sub(r"@[^@]*@", "c", stmt)
    n = t.count("hot_rsqrt(")
    for op in ("+=", "-=", "*="):
        n += t.count(op)
        t = t.replace(op, " = ")
    prev = ""
    for ch in t:
        if ch in "*+-":
            if not (ch == "-" and prev in "(=,"):
                n += 1
        if not ch.isspace():
            prev = ch
    return n


def m2p_source_flops(p):
    """Operation count of the shipped m2p_eval<p> statements (the Horner form), FMA = 2."""
    L, _ = _eval_stmts(p)
    return sum(_count_ops(st) for st in L)


class _Prog:
    """Straight-line code in SSA form built from steps v = a + m * b (one fused
    multiply-add), m one of the Horner variables y100, y010, y001.  Operands are
    variable names, coefficient references ('@...@', constant) or None (zero).  With
    tangent, every variable v gets dv = da + dm b + m db, the forward-mode derivative
    along (dy100, dy010, dy001)."""

    def __init__(self, tangent):
        self.L = []
        self.tangent = tangent
        self.var = set()

    def d(self, x):
        return "d" + x if x in self.var else None

    def fma(self, name, a, m, b):
        if b is None:
            return a
        self.L.append(f"const T {name} = " + (f"{m} * {b};" if a is None else f"{a} + {m} * {b};"))
        self.var.add(name)
        if self.tangent:
            terms = [t for t in (self.d(a) if a is not None else None, f"d{m} * {b}",
                                 f"{m} * {self.d(b)}" if self.d(b) else None) if t]
            self.L.append(f"const T d{name} = " + " + ".join(terms) + ";")
        return name


def _horner_grad(P, X, n, ref, hess=False):
    """The polynomial X(y) = sum_{|g| <= n} c_g y^g and its gradient from the
    coefficients c_g alone: nested Horner in y_z (inner), y_y, y_x (outer), each chain
    carrying its derivative in its own variable (d <- d y + h before h <- h y + c), and
    the y_z- and y_y-derivatives of the inner chains carried through the outer ones.
    With hess, the second derivatives as well: a second-derivative chain e <- e y + d
    (before d is updated) gives half the pure second derivative, a derivative chain over
    an outer variable of a carried first derivative gives the mixed one.
    Returns the names of X, dX/dy_x, dX/dy_y, dX/dy_z and, with hess, of X_xx/2, X_xy,
    X_xz, X_yy/2, X_yz, X_zz/2 (None where identically zero)."""
    f = P.fma
    S = Sx = Sy = Sz = None
    Sxxh = Sxy = Sxz = Syyh = Syz = Szzh = None
    for i in range(n, -1, -1):
        t = ty = tz = tyyh = tyz = tzzh = None
        for j in range(n - i, -1, -1):
            m = n - i - j
            h, hz, hzzh = ref(i, j, m), None, None
            for l in range(m - 1, -1, -1):
                if hess:
                    hzzh = f(f"hzz{X}_{i}_{j}_{l}", hz, "y001", hzzh)
                hz = h if hz is None else f(f"hz{X}_{i}_{j}_{l}", h, "y001", hz)
                h = f(f"h{X}_{i}_{j}_{l}", ref(i, j, l), "y001", h)
            if t is None:
                t, tz, tzzh = h, hz, hzzh
            else:
                if hess:
                    tyyh = f(f"tyy{X}_{i}_{j}", ty, "y010", tyyh)
                    tyz = f(f"tyz{X}_{i}_{j}", tz, "y010", tyz)
                    tzzh = f(f"tzz{X}_{i}_{j}", hzzh, "y010", tzzh)
                ty = t if ty is None else f(f"ty{X}_{i}_{j}", t, "y010", ty)
                t = f(f"t{X}_{i}_{j}", h, "y010", t)
                tz = hz if tz is None else f(f"tz{X}_{i}_{j}", hz, "y010", tz)
        if S is None:
            S, Sy, Sz, Syyh, Syz, Szzh = t, ty, tz, tyyh, tyz, tzzh
        else:
            if hess:
                Sxxh = f(f"sxx{X}_{i}", Sx, "y100", Sxxh)
                Sxy = f(f"sxy{X}_{i}", Sy, "y100", Sxy)
                Sxz = f(f"sxz{X}_{i}", Sz, "y100", Sxz)
                Syyh = f(f"syy{X}_{i}", tyyh, "y100", Syyh)
                Syz = f(f"syz{X}_{i}", tyz, "y100", Syz)
                Szzh = f(f"szz{X}_{i}", tzzh, "y100", Szzh)
            Sx = S if Sx is None else f(f"sx{X}_{i}", S, "y100", Sx)
            S = f(f"s{X}_{i}", t, "y100", S)
            Sy = ty if Sy is None else f(f"sy{X}_{i}", ty, "y100", Sy)
            Sz = tz if Sz is None else f(f"sz{X}_{i}", tz, "y100", Sz)
    out = [S, Sx, Sy, Sz]
    if hess:
        out += [Sxxh, Sxy, Sxz, Syyh, Syz, Szzh]
    return out


def _horner_w(dst, names, tangent):
    """dst = names[0] + w (names[1] + w (...)), with its tangent when asked."""
    out = []

    def dn(nm):
        return "T(0)" if nm.startswith("T(") else "d" + nm

    t, dt = names[-1], dn(names[-1])
    for q, nm in enumerate(reversed(names[:-1])):
        v = f"w{dst}_{q}"
        out.append(f"const T {v} = {nm} + w * {t};")
        if tangent:
            out.append(f"const T d{v} = {dn(nm)} + dw * {t} + w * {dt};")
        t, dt = v, "d" + v
    out.append(f"const T {dst} = {t};")
    if tangent:
        out.append(f"const T d{dst} = {dt};")
    return out


def _eval_stmts(p, tangent=False):
    """Statements of one M2P interaction with symbolic coefficient references
    ('@S,k,i,j,l@' for C_{b,k}, b = (i, j, l)), and the flop convention.
    Phi = rho sum_k w^k S_k(y); the gradient needs dS_k/dy_d, formed alongside S_k by
    the derivative-carrying Horner chains of _horner_grad, and Q = sum_k w^k sum_n
    (1+2k+2n) S_{k,n}, which by Euler's theorem for the degree-n parts is sum_k w^k
    [(1+2k) S_k + 2 y . grad S_k].  With tangent, the forward-mode derivative along the
    input direction (ux, uy, uz) is carried alongside: (d a / d R) u, the Hessian of the
    expansion applied to u."""
    L = ["rx *= is; ry *= is; rz *= is;"]
    if tangent:
        L.append("const T drx = ux * is, dry = uy * is, drz = uz * is;")
    # from e2 up, so that the sum is three fused multiply-adds
    L.append("const T u = e2 + rx * rx + ry * ry + rz * rz;")
    if tangent:
        L.append("const T du = T(2) * (rx * drx + ry * dry + rz * drz);")
    L.append("const T rho = hot_rsqrt(u);")
    L.append("const T w = rho * rho;")
    if tangent:
        L.append("const T drho = T(-0.5) * rho * w * du;")
        L.append("const T dw = T(2) * rho * drho;")
    L.append(f"const T {mname((1,0,0))} = rx * w, {mname((0,1,0))} = ry * w, {mname((0,0,1))} = rz * w;")
    if tangent:
        L.append("const T dy100 = drx * w + rx * dw, dy010 = dry * w + ry * dw, dy001 = drz * w + rz * dw;")
    K = p // 2
    for k in range(K + 1):
        n = p - 2 * k
        # with tangent, the Hessian of S_k applied to dy gives the tangents of the gradient
        # (no forward-mode chains)
        P = _Prog(False)
        names = _horner_grad(P, f"S{k}", n, lambda i, j, l, k=k: f"@S,{k},{i},{j},{l}@", hess=tangent)
        L += P.L
        for nm, v in zip([f"S{k}", f"G{k}_0", f"G{k}_1", f"G{k}_2"], names[:4]):
            L.append(f"const T {nm} = {v if v is not None else 'T(0)'};")
        if tangent:
            dy = ("dy100", "dy010", "dy001")

            def lin(terms):
                t = [f"{c}{a} * {b}" for c, a, b in terms if a is not None]
                return " + ".join(t) if t else "T(0)"
            L.append(f"const T dS{k} = " + lin([("", f"G{k}_{d}", dy[d]) for d in range(3)]) + ";")
            hxx, hxy, hxz, hyy, hyz, hzz = names[4:]
            hm = [[(hxx, "T(2) * "), (hxy, ""), (hxz, "")],
                  [(hxy, ""), (hyy, "T(2) * "), (hyz, "")],
                  [(hxz, ""), (hyz, ""), (hzz, "T(2) * ")]]
            for d in range(3):
                L.append(f"const T dG{k}_{d} = " + lin([(c, a, dy[e]) for e, (a, c) in enumerate(hm[d])]) + ";")
        if n >= 1:
            L.append(f"const T yg{k} = y100 * G{k}_0 + y010 * G{k}_1 + y001 * G{k}_2;")
            if tangent:
                L.append(f"const T dyg{k} = dy100 * G{k}_0 + y100 * dG{k}_0 + dy010 * G{k}_1 + y010 * dG{k}_1 + "
                         f"dy001 * G{k}_2 + y001 * dG{k}_2;")
            L.append(f"const T Q{k} = T({1 + 2 * k}) * S{k} + T(2) * yg{k};")
            if tangent:
                L.append(f"const T dQ{k} = T({1 + 2 * k}) * dS{k} + T(2) * dyg{k};")
        else:
            L.append(f"const T Q{k} = T({1 + 2 * k}) * S{k};")
            if tangent:
                L.append(f"const T dQ{k} = T({1 + 2 * k}) * dS{k};")
    L += _horner_w("S", [f"S{k}" for k in range(K + 1)], tangent)
    L += _horner_w("Q", [f"Q{k}" for k in range(K + 1)], tangent)
    for d in range(3):
        ks = [k for k in range(K + 1) if p - 2 * k >= 1]
        if ks:
            L += _horner_w(f"Gs{d}", [f"G{k}_{d}" for k in range(max(ks) + 1)], tangent)
        else:
            L.append(f"const T Gs{d} = T(0);")
            if tangent:
                L.append(f"const T dGs{d} = T(0);")
    L.append("phi -= rho * S;")
    if tangent:
        L.append("const T rs = rho * is;")
        L.append("const T drs = drho * is;")
        for d, (yn, an) in enumerate(((mname((1,0,0)), "ax"), (mname((0,1,0)), "ay"), (mname((0,0,1)), "az"))):
            L.append(f"{an} += rs * (w * Gs{d} - {yn} * Q);")
            L.append(f"d{an} += drs * (w * Gs{d} - {yn} * Q) + rs * (dw * Gs{d} + w * dGs{d} - d{yn} * Q - "
                     f"{yn} * dQ);")
    else:
        # w Gs - y Q = w (Gs - R Q) (y = R w): the common factor rho inv_s w once, then two
        # fused multiply-adds per component
        L.append("const T rsw = rho * is * w;")
        for d, (rn, an) in enumerate((("rx", "ax"), ("ry", "ay"), ("rz", "az"))):
            L.append(f"{an} += rsw * (Gs{d} - {rn} * Q);")
    return L, M2P_FLOP_CONVENTION[p]


def gen_tangent(p):
    L, _ = _eval_stmts(p, tangent=True)
    slot = layout(p)
    out = []
    for T, VEC, VW, suf in (("float", "float4", 4, "f32"), ("double", "double2", 2, "f64")):
        comp = "xyzw"
        code = [f"__device__ __forceinline__ void m2p_tangent_{p}_{suf}(const {T}* __restrict__ c, {T} rx, {T} ry, "
                f"{T} rz, {T} ux, {T} uy, {T} uz, {T}& phi, {T}& ax, {T}& ay, {T}& az, {T}& dax, {T}& day, "
                f"{T}& daz) {{",
                f"  using T = {T};",
                f"  const {VEC}* __restrict__ cv = reinterpret_cast<const {VEC}*>(c);"]
        loaded = set()

        def need(g):
            if g not in loaded:
                loaded.add(g)
                code.append(f"  const {VEC} v{g} = cv[{g}];")

        need(0)
        code.append("  const T is = v0.x, e2 = v0.y;")
        for st in L:
            parts = st.split("@")
            for i in range(1, len(parts), 2):
                sl = slot[parts[i]]
                g = sl // VW
                need(g)
                parts[i] = f"v{g}.{comp[sl % VW]}"
            code.append("  " + "".join(parts))
        code.append("}")
        out.append("\n".join(code))
    return "\n".join(out)


def gen_cbar(p):
    """Adjoint of one interaction with respect to the record coefficients C_{b,k}
    (the accelerations and potential are linear in them): with output weights u (for
    the acceleration) and v (for the potential),
        dL/dC_{b,k} = A_{k,n} y^b + B_k D_u(y^b),
        A_{k,n} = -w^k (v rho + rs (1+2k+2n) (u.y)),   B_k = rs w^{k+1},
    D_u(y^b) = sum_d u_d b_d y^{b-e_d}; accumulated into cb[] in s_terms order."""
    S = s_terms(p)
    K = p // 2
    out = []
    for T, suf in (("float", "f32"), ("double", "f64")):
        L = [f"__device__ __forceinline__ void m2p_cbar_{p}_{suf}({T} is, {T} e2, {T} rx, {T} ry, {T} rz, "
             f"{T} ux, {T} uy, {T} uz, {T} v, {T}* __restrict__ cb) {{",
             f"  using T = {T};",
             "  rx *= is; ry *= is; rz *= is;",
             "  const T u = rx * rx + ry * ry + rz * rz + e2;",
             "  const T rho = hot_rsqrt(u);",
             "  const T w = rho * rho;",
             "  const T rs = rho * is;",
             "  const T y100 = rx * w, y010 = ry * w, y001 = rz * w;",
             "  const T Dy100 = ux, Dy010 = uy, Dy001 = uz;",
             "  const T uy_ = ux * y100 + uy * y010 + uz * y001;",
             "  const T y000 = T(1), Dy000 = T(0);",
             "  T wk[%d];" % (K + 2),
             "  wk[0] = T(1);",
             f"  for (int q = 1; q < {K + 2}; ++q) wk[q] = wk[q - 1] * w;"]
        # A_{k,n} = a_k + n b_k with a_k = -w^k (v rho + rs (1+2k) u.y), b_k = -2 w^k rs u.y
        for k in range(K + 1):
            L.append(f"  const T B{k} = rs * wk[{k + 1}];")
            L.append(f"  const T a{k} = -wk[{k}] * (v * rho + rs * T({1 + 2 * k}) * uy_);")
            L.append(f"  const T b{k} = T(-2) * wk[{k}] * rs * uy_;")
        sidx = {(k, n, b): i for i, (k, n, b) in enumerate(S)}
        # degree by degree: the monomials of degree n (and their derivatives along u) are
        # formed from those of degree n-1 and consumed at once, so that only two degrees
        # are live together
        for n in range(0, p + 1):
            if n >= 2:
                for a in midx(n)[ncomp(n - 1):]:
                    d = 0 if a[0] > 0 else (1 if a[1] > 0 else 2)
                    prev = list(a)
                    prev[d] -= 1
                    prev = mname(tuple(prev))
                    unit = [mname((1, 0, 0)), mname((0, 1, 0)), mname((0, 0, 1))][d]
                    ud = ["ux", "uy", "uz"][d]
                    L.append(f"  const T {mname(a)} = {prev} * {unit};")
                    L.append(f"  const T D{mname(a)} = D{prev} * {unit} + {prev} * {ud};")
            for k in range(K + 1):
                if n > p - 2 * k:
                    continue
                L.append(f"  const T A{k}_{n} = a{k} + T({n}) * b{k};")
                # two separate accumulations, each one fused multiply-add (a single
                # expression would be evaluated as multiply, multiply-add and add)
                for b in (midx(n)[ncomp(n - 1):] if n > 0 else [(0, 0, 0)]):
                    i = sidx[(k, n, b)]
                    if n > 0:
                        L.append(f"  cb[{i}] += A{k}_{n} * {mname(b)};")
                        L.append(f"  cb[{i}] += B{k} * D{mname(b)};")
                    else:
                        L.append(f"  cb[{i}] += A{k}_{n};")
        L.append("}")
        out.append("\n".join(L))
    return "\n".join(out)


def gen_record_adjoint(p):
    """Transpose of the moments -> coefficients map of m2p_record: given dL/dC_{b,k}
    (s_terms order), accumulate dL/dM_a (FP64)."""
    S = s_terms(p)
    idx = {a: i for i, a in enumerate(midx(p))}
    L = [f"__device__ __forceinline__ void m2p_record_adjoint_{p}(const double* __restrict__ cb, double inv_s, "
         "double G, double* __restrict__ Mbar) {",
         f"  double ip[{2 * p + 2}];",
         "  ip[0] = 1.0;",
         f"  for (int q = 1; q < {2 * p + 2}; ++q) ip[q] = ip[q - 1] * inv_s;"]
    for i, (k, n, b) in enumerate(S):
        m = n + k
        const = (-1) ** k * dfact(2 * m - 1) / (2 ** k * fact3(b))
        L.append(f"  {{ const double t = G * ip[{1 + 2 * k + n}] * {const!r} * cb[{i}];")
        for l in midx(k)[ncomp(k - 1) if k > 0 else 0:]:
            a = add(b, (2 * l[0], 2 * l[1], 2 * l[2]))
            L.append(f"    Mbar[{idx[a]}] += t * {1.0 / fact3(l)!r};")
        L.append("  }")
    L.append("}")
    return "\n".join(L)


def record_adjoint_table(p):
    """The map of gen_record_adjoint gathered per moment a: dL/dM_a = G sum_j f_j inv_s^e_j
    dL/dC[q_j], terms in statement order.  Returns (start[ncomp+1], q, e, f)."""
    S = s_terms(p)
    idx = {a: i for i, a in enumerate(midx(p))}
    terms = [[] for _ in range(ncomp(p))]
    for i, (k, n, b) in enumerate(S):
        m = n + k
        const = (-1) ** k * dfact(2 * m - 1) / (2 ** k * fact3(b))
        for l in midx(k)[ncomp(k - 1) if k > 0 else 0:]:
            a = add(b, (2 * l[0], 2 * l[1], 2 * l[2]))
            terms[idx[a]].append((i, 1 + 2 * k + n, const * (1.0 / fact3(l))))
    start, q, e, f = [0], [], [], []
    for t in terms:
        for (i, ee, ff) in t:
            q.append(i)
            e.append(ee)
            f.append(ff)
        start.append(len(q))
    return start, q, e, f


def m2m_transposed(p):
    """For each b: the pairs (a >= b, C(a,b), g = a - b) of the translation, so that
    dL/dM_b(child) += sum_a C(a,b) (z_child - z_parent)^{a-b} dL/dM_a(parent)."""
    ia = midx(p)
    idx = {a: i for i, a in enumerate(ia)}
    start, aidx, gidx, coef = [], [], [], []
    for b in ia:
        start.append(len(aidx))
        for a in ia:
            if all(b[d] <= a[d] for d in range(3)):
                g = (a[0] - b[0], a[1] - b[1], a[2] - b[2])
                aidx.append(idx[a])
                gidx.append(idx[g])
                coef.append(math.comb(a[0], b[0]) * math.comb(a[1], b[1]) * math.comb(a[2], b[2]))
    start.append(len(aidx))
    return start, aidx, gidx, coef


def layout(p):
    """Record slots in the order the interaction code first reads them, so that vector
    loads stay close to their use.  Slots 0..7 hold the header: inv_s, eps^2/s^2, and the
    cell centre as a hi/lo pair (hi = centre rounded to T, lo = the rounding remainder)."""
    L, _ = _eval_stmts(p)
    order = []
    seen = set()
    for st in L:
        parts = st.split("@")
        for i in range(1, len(parts), 2):
            key = parts[i]
            if key not in seen:
                seen.add(key)
                order.append(key)
    return {key: HDR + i for i, key in enumerate(order)}


def gen_eval(p):
    """Two specialisations: float (float4 loads) and double (double2 loads).  The routine
    proper, m2p_eval_s, takes R already scaled by the record's inv_s (R/s, which a caller
    holding x and the scaled centre offset forms with one fused multiply-add per axis,
    exactly: the scale is a power of two); m2p_eval scales R and calls it."""
    L, fl = _eval_stmts(p)
    assert L[0] == "rx *= is; ry *= is; rz *= is;"
    L = L[1:]
    slot = layout(p)
    out = []
    for T, VEC, VW, suf in (("float", "float4", 4, "f32"), ("double", "double2", 2, "f64")):
        comp = "xyzw"
        code = [f"__device__ __forceinline__ void m2p_eval_s_{p}_{suf}(const {T}* __restrict__ c, {T} rx, {T} ry, "
                f"{T} rz, {T}& phi, {T}& ax, {T}& ay, {T}& az) {{",
                f"  using T = {T};",
                f"  const {VEC}* __restrict__ cv = reinterpret_cast<const {VEC}*>(c);"]
        loaded = set()

        def need(g):
            if g not in loaded:
                loaded.add(g)
                code.append(f"  const {VEC} v{g} = cv[{g}];")

        need(0)
        if VW == 2:
            code.append("  const T is = v0.x, e2 = v0.y;")
        else:
            code.append("  const T is = v0.x, e2 = v0.y;")
        for st in L:
            parts = st.split("@")
            for i in range(1, len(parts), 2):
                sl = slot[parts[i]]
                g = sl // VW
                need(g)
                parts[i] = f"v{g}.{comp[sl % VW]}"
            code.append("  " + "".join(parts))
        code.append("}")
        code.append(f"__device__ __forceinline__ void m2p_eval_{p}_{suf}(const {T}* __restrict__ c, {T} rx, {T} ry, "
                    f"{T} rz, {T}& phi, {T}& ax, {T}& ay, {T}& az) {{")
        code.append(f"  const {T} is = c[0];")
        code.append(f"  m2p_eval_s_{p}_{suf}(c, rx * is, ry * is, rz * is, phi, ax, ay, az);")
        code.append("}")
        out.append("\n".join(code))
    return "\n".join(out), len(s_terms(p)), fl


def gen_record(p):
    """Raw moments -> scaled traced coefficients (FP64 arithmetic), in record order."""
    S = s_terms(p)
    ns = len(S)
    slot = layout(p)
    idx = {a: i for i, a in enumerate(midx(p))}
    L = []
    L.append(f"template <typename T> __device__ __forceinline__ void m2p_record_{p}("
             "const double* __restrict__ M, const double* __restrict__ z, double inv_s, double G, double eps, "
             "T* __restrict__ rec) {")
    L.append(f"  double ip[{p + 2 + p}];")
    L.append("  ip[0] = 1.0;")
    L.append(f"  for (int q = 1; q < {2 * p + 2}; ++q) ip[q] = ip[q - 1] * inv_s;")
    L.append("  rec[0] = T(inv_s); rec[1] = T((eps * inv_s) * (eps * inv_s));")
    L.append("  for (int d = 0; d < 3; ++d) { const T hi = T(z[d]); rec[2 + d] = hi; rec[5 + d] = T(z[d] - double(hi)); }")
    L.append(f"  double C[{ns}];")
    for i, (k, n, b) in enumerate(S):
        m = n + k
        const = (-1) ** k * dfact(2 * m - 1) / (2 ** k * fact3(b))
        terms = []
        for l in midx(k)[ncomp(k - 1) if k > 0 else 0:]:
            a = add(b, (2 * l[0], 2 * l[1], 2 * l[2]))
            terms.append(f"M[{idx[a]}] * {1.0 / fact3(l)!r}")
        L.append(f"  C[{i}] = G * ip[{1 + 2 * k + n}] * {const!r} * (" + " + ".join(terms) + ");")
        L.append(f"  rec[{slot[f'S,{k},{b[0]},{b[1]},{b[2]}']}] = T(C[{i}]);")
    rl = (HDR + ns + 3) // 4 * 4
    for q in range(HDR + ns, rl):
        L.append(f"  rec[{q}] = T(0);")
    L.append("}")
    return "\n".join(L)


def main(out_path):
    parts = []
    parts.append("// Generated by gen_kernels.py -- do not edit by hand.\n#pragma once\n")
    parts.append(f"#define HOT_PMAX {PMAX}")
    parts.append(f"#define HOT_NCOMP_MAX {ncomp(PMAX)}")
    recl, fll = [], []
    evals, records = [], []
    for p in range(PMAX + 1):
        code, ns, fl = gen_eval(p)
        evals.append(code)
        records.append(gen_record(p))
        recl.append((HDR + ns + 3) // 4 * 4)
        fll.append(fl)
    parts.append("static constexpr int HOT_REC_LEN[%d] = {%s};" % (PMAX + 1, ", ".join(map(str, recl))))
    parts.append("static constexpr int M2P_FLOPS[%d] = {%s};" % (PMAX + 1, ", ".join(map(str, fll))))
    parts.append("static constexpr int HOT_NCOMP[%d] = {%s};" % (PMAX + 1, ", ".join(str(ncomp(p)) for p in range(PMAX + 1))))
    # multi-index table (order PMAX covers every lower order as a prefix)
    ia = midx(PMAX)
    parts.append("__device__ __constant__ unsigned char hot_midx[%d][3] = {%s};" % (
        len(ia), ", ".join("{%d,%d,%d}" % a for a in ia)))
    parts.extend(evals)
    parts.extend(records)
    ts, ta, tg, tc = m2m_transposed(ADJ_PMAX)
    parts.append(f"__device__ const unsigned short m2mt_start[{len(ts)}] = {{{', '.join(map(str, ts))}}};")
    parts.append(f"__device__ const unsigned char m2mt_alpha[{len(ta)}] = {{{', '.join(map(str, ta))}}};")
    parts.append(f"__device__ const unsigned char m2mt_gamma[{len(tg)}] = {{{', '.join(map(str, tg))}}};")
    parts.append(f"__device__ const double m2mt_coef[{len(tc)}] = {{{', '.join(repr(float(c)) for c in tc)}}};")
    parts.append("static constexpr int HOT_NS[%d] = {%s};" % (PMAX + 1, ", ".join(str(len(s_terms(q))) for q in range(PMAX + 1))))
    # record-adjoint gather tables of every order, concatenated (per-order bases)
    sb, eb, rs, rq, re_, rf = [], [], [], [], [], []
    for q in range(ADJ_PMAX + 1):
        st, qq, ee, ff = record_adjoint_table(q)
        sb.append(len(rs))
        eb.append(len(rq))
        rs.extend(x + len(rq) for x in st)
        rq.extend(qq)
        re_.extend(ee)
        rf.extend(ff)
    parts.append(f"#define HOT_ADJ_PMAX {ADJ_PMAX}")
    parts.append("static constexpr int RADJ_SBASE[%d] = {%s};" % (ADJ_PMAX + 1, ", ".join(map(str, sb))))
    parts.append(f"__device__ const unsigned short radj_start[{len(rs)}] = {{{', '.join(map(str, rs))}}};")
    parts.append(f"__device__ const unsigned short radj_q[{len(rq)}] = {{{', '.join(map(str, rq))}}};")
    parts.append(f"__device__ const unsigned char radj_e[{len(re_)}] = {{{', '.join(map(str, re_))}}};")
    parts.append(f"__device__ const double radj_f[{len(rf)}] = {{{', '.join(repr(float(x)) for x in rf)}}};")
    for q in range(ADJ_PMAX + 1):
        parts.append(gen_tangent(q))
        parts.append(gen_cbar(q))
        parts.append(gen_record_adjoint(q))
    tw = ["template <int P, typename T> __device__ __forceinline__ void m2p_tangent(const T* __restrict__ c, "
          "T rx, T ry, T rz, T ux, T uy, T uz, T& phi, T& ax, T& ay, T& az, T& dax, T& day, T& daz) {"]
    cw = ["template <int P, typename T> __device__ __forceinline__ void m2p_cbar(T is, T e2, T rx, T ry, T rz, "
          "T ux, T uy, T uz, T v, T* __restrict__ cb) {"]
    aw = ["template <int P> __device__ __forceinline__ void m2p_record_adjoint(const double* __restrict__ cb, "
          "double inv_s, double G, double* __restrict__ Mbar) {"]
    for q in range(ADJ_PMAX + 1):
        kw = "if" if q == 0 else "else if"
        tw.append(f"  {kw} constexpr (P == {q}) {{ if constexpr (sizeof(T) == 4) m2p_tangent_{q}_f32(c, rx, ry, rz, ux, uy, uz, "
                  f"phi, ax, ay, az, dax, day, daz); else m2p_tangent_{q}_f64(c, rx, ry, rz, ux, uy, uz, phi, ax, ay, az, "
                  f"dax, day, daz); }}")
        cw.append(f"  {kw} constexpr (P == {q}) {{ if constexpr (sizeof(T) == 4) m2p_cbar_{q}_f32(is, e2, rx, ry, rz, "
                  f"ux, uy, uz, v, cb); else m2p_cbar_{q}_f64(is, e2, rx, ry, rz, ux, uy, uz, v, cb); }}")
        aw.append(f"  {kw} constexpr (P == {q}) m2p_record_adjoint_{q}(cb, inv_s, G, Mbar);")
    for w_ in (tw, cw, aw):
        w_.append("}")
        parts.append("\n".join(w_))
    es = ["template <int P, typename T> __device__ __forceinline__ void m2p_eval_s("
          "const T* __restrict__ c, T rx, T ry, T rz, T& phi, T& ax, T& ay, T& az) {"]
    ev = ["template <int P, typename T> __device__ __forceinline__ void m2p_eval("
          "const T* __restrict__ c, T rx, T ry, T rz, T& phi, T& ax, T& ay, T& az) {"]
    rc = ["template <int P, typename T> __device__ __forceinline__ void m2p_record("
          "const double* __restrict__ M, const double* __restrict__ z, double inv_s, double G, double eps, "
          "T* __restrict__ rec) {"]
    for p in range(PMAX + 1):
        kw = "if" if p == 0 else "else if"
        ev.append(f"  {kw} constexpr (P == {p}) {{ if constexpr (sizeof(T) == 4) m2p_eval_{p}_f32(c, rx, ry, rz, phi, ax, ay, az); "
                  f"else m2p_eval_{p}_f64(c, rx, ry, rz, phi, ax, ay, az); }}")
        es.append(f"  {kw} constexpr (P == {p}) {{ if constexpr (sizeof(T) == 4) m2p_eval_s_{p}_f32(c, rx, ry, rz, phi, ax, ay, "
                  f"az); else m2p_eval_s_{p}_f64(c, rx, ry, rz, phi, ax, ay, az); }}")
        rc.append(f"  {kw} constexpr (P == {p}) m2p_record_{p}<T>(M, z, inv_s, G, eps, rec);")
    ev.append("}")
    es.append("}")
    rc.append("}")
    parts.append("\n".join(es))
    parts.append("\n".join(ev))
    parts.append("\n".join(rc))
    src = "\n".join(parts) + "\n"
    with open(out_path, "w") as f:
        f.write(src)
    return recl, fll


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "generated.cuh")
    recl, fll = main(out)
    print("record lengths", recl)
    print("flops per M2P", fll)
