"""Generator of the per-angular-momentum-class ERI device code (run by the build).

For every canonical class (la lb | lc ld) of s/p/d shells (la >= lb, lc >= ld,
bra pair class >= ket pair class: 21 classes) it emits a traits struct with

  vrr<R>(G, geo, acc)   Obara-Saika / Head-Gordon-Pople vertical recursion for
                        one primitive quartet: builds [e0|f0]^(0) for
                        |e| in [la, la+lb], |f| in [lc, lc+ld] from the
                        auxiliary integrals G_m = [00|00]^(m), m = 0..L, and
                        adds them into the contracted accumulators acc.
  hrr<R>(acc, AB, CD, out)
                        horizontal recursion on the contracted integrals,
                        (a,b+1_i| = (a+1_i,b| + AB_i (a,b|, first on the bra
                        then on the ket, giving (ab|cd) in Cartesian order.

Everything is straight-line code (one local per recursion node), so the
compiler keeps it in registers where it can.  The emitted flop counts (every
multiply and add as written) are exported per class for roofline accounting.

Recursions (Obara & Saika 1986; Head-Gordon & Pople 1988), with
PA = P - A, QC = Q - C, WP = W - P = -(rho/p) PQ, WQ = W - Q = (rho/q) PQ:
  [e+1_i|0]^(m) = PA_i [e|0]^(m) + WP_i [e|0]^(m+1)
                  + e_i/(2p) ([e-1_i|0]^(m) - rho/p [e-1_i|0]^(m+1))
  [e|f+1_i]^(m) = QC_i [e|f]^(m) + WQ_i [e|f]^(m+1)
                  + f_i/(2q) ([e|f-1_i]^(m) - rho/q [e|f-1_i]^(m+1))
                  + e_i/(2(p+q)) [e-1_i|f]^(m+1)
The same recursion holds for the erf/erfc-attenuated kernels once the G_m are
the attenuated auxiliary integrals.
"""
from __future__ import annotations

import os
import sys

LMAX = 2
PAIR_CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]  # ss ps pp ds dp dd


def comps(l):
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def comps_range(lo, hi):
    out = []
    for l in range(lo, hi + 1):
        out.extend(comps(l))
    return out


def quartet_classes():
    out = []
    for ib, (la, lb) in enumerate(PAIR_CLASSES):
        for ik, (lc, ld) in enumerate(PAIR_CLASSES):
            if ik <= ib:
                out.append((ib, ik, la, lb, lc, ld))
    return out


def _sub(v, i, k=1):
    w = list(v)
    w[i] -= k
    return tuple(w)


def _add(v, i, k=1):
    w = list(v)
    w[i] += k
    return tuple(w)


def _nm(v):
    return "".join(str(x) for x in v)


AX = "xyz"
# classes with more contracted accumulators than this get out-of-line
# recursion functions (their working set lives in local memory anyway)
INLINE_MAX_ACC = 160


class VRR:
    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.L = la + lb + lc + ld
        self.E = comps_range(la, la + lb)
        self.F = comps_range(lc, lc + ld)
        self.names = {}
        self.lines = []
        self.flops = 0

    def node(self, e, f, m):
        key = (e, f, m)
        if key in self.names:
            return self.names[key]
        if sum(e) == 0 and sum(f) == 0:
            name = f"G[{m}]"
            self.names[key] = name
            return name
        terms = []
        fl = 0
        if sum(f) > 0:
            i = next(k for k in range(3) if f[k] > 0)
            f1 = _sub(f, i)
            terms.append(f"QC{AX[i]} * {self.node(e, f1, m)}")
            terms.append(f"WQ{AX[i]} * {self.node(e, f1, m + 1)}")
            fl += 2
            if f1[i] > 0:
                f2 = _sub(f1, i)
                a, b = self.node(e, f2, m), self.node(e, f2, m + 1)
                terms.append(f"R({f1[i]}) * oo2q * ({a} - roq * {b})")
                fl += 3 + (f1[i] > 1)
            if e[i] > 0:
                terms.append(f"R({e[i]}) * oo2pq * {self.node(_sub(e, i), f1, m + 1)}")
                fl += 1 + (e[i] > 1)
        else:
            i = next(k for k in range(3) if e[k] > 0)
            e1 = _sub(e, i)
            terms.append(f"PA{AX[i]} * {self.node(e1, f, m)}")
            terms.append(f"WP{AX[i]} * {self.node(e1, f, m + 1)}")
            fl += 2
            if e1[i] > 0:
                e2 = _sub(e1, i)
                a, b = self.node(e2, f, m), self.node(e2, f, m + 1)
                terms.append(f"R({e1[i]}) * oo2p * ({a} - rop * {b})")
                fl += 3 + (e1[i] > 1)
        fl += len(terms) - 1
        self.flops += fl
        name = f"v{_nm(e)}_{_nm(f)}_{m}"
        self.names[key] = name
        self.lines.append(f"    const R {name} = " + " + ".join(terms) + ";")
        return name

    def emit(self):
        acc_lines = []
        nf = len(self.F)
        for ie, e in enumerate(self.E):
            for jf, f in enumerate(self.F):
                nm = self.node(e, f, 0)
                acc_lines.append(f"    acc[{ie * nf + jf}] += {nm};")
                self.flops += 1
        return self.lines + acc_lines


class HRR:
    """Contracted horizontal recursion, bra then ket."""

    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.E = comps_range(la, la + lb)
        self.F = comps_range(lc, lc + ld)
        self.eidx = {e: i for i, e in enumerate(self.E)}
        self.fidx = {f: i for i, f in enumerate(self.F)}
        self.lines = []
        self.flops = 0

    def emit(self):
        la, lb, lc, ld = self.la, self.lb, self.lc, self.ld
        nf = len(self.F)
        # bra: (a b | f] for every f
        bra = {}

        def bnode(a, b, jf):
            key = (a, b, jf)
            if key in bra:
                return bra[key]
            if sum(b) == 0:
                nm = f"acc[{self.eidx[a] * nf + jf}]"
            else:
                i = next(k for k in range(3) if b[k] > 0)
                b1 = _sub(b, i)
                x = bnode(_add(a, i), b1, jf)
                y = bnode(a, b1, jf)
                nm = f"h{_nm(a)}_{_nm(b)}_{jf}"
                self.lines.append(f"    const R {nm} = {x} + AB{AX[i]} * {y};")
                self.flops += 2
            bra[key] = nm
            return nm

        A, B, C, D = comps(la), comps(lb), comps(lc), comps(ld)
        ket = {}

        def knode(ia, ib, c, d):
            key = (ia, ib, c, d)
            if key in ket:
                return ket[key]
            if sum(d) == 0:
                nm = bnode(A[ia], B[ib], self.fidx[c])
            else:
                i = next(k for k in range(3) if d[k] > 0)
                d1 = _sub(d, i)
                x = knode(ia, ib, _add(c, i), d1)
                y = knode(ia, ib, c, d1)
                nm = f"k{ia}_{ib}_{_nm(c)}_{_nm(d)}"
                self.lines.append(f"    const R {nm} = {x} + CD{AX[i]} * {y};")
                self.flops += 2
            ket[key] = nm
            return nm

        nB, nC, nD = len(B), len(C), len(D)
        outs = []
        for ia in range(len(A)):
            for ib in range(nB):
                for ic, c in enumerate(C):
                    for id_, d in enumerate(D):
                        nm = knode(ia, ib, c, d)
                        outs.append(f"    out[{((ia * nB + ib) * nC + ic) * nD + id_}] = {nm};")
        return self.lines + outs


def gen_class(ib, ik, la, lb, lc, ld):
    v = VRR(la, lb, lc, ld)
    vl = v.emit()
    h = HRR(la, lb, lc, ld)
    hl = h.emit()
    name = f"Cls{la}{lb}{lc}{ld}"
    NA, NB, NC, ND = (len(comps(x)) for x in (la, lb, lc, ld))
    src = []
    src.append(f"struct {name} {{")
    src.append(f"  static constexpr int la = {la}, lb = {lb}, lc = {lc}, ld = {ld};")
    src.append(f"  static constexpr int bra_class = {ib}, ket_class = {ik};")
    src.append(f"  static constexpr int L = {la + lb + lc + ld};")
    src.append(f"  static constexpr int NA = {NA}, NB = {NB}, NC = {NC}, ND = {ND};")
    src.append(f"  static constexpr int NE = {len(v.E)}, NF = {len(v.F)}, NACC = {len(v.E) * len(v.F)};")
    src.append(f"  static constexpr int NOUT = {NA * NB * NC * ND};")
    src.append(f"  static constexpr int VRR_FLOPS = {v.flops}, HRR_FLOPS = {h.flops};")
    inl = "__forceinline__" if len(v.E) * len(v.F) <= INLINE_MAX_ACC else "__noinline__"
    src.append("  template <typename R>")
    src.append(f"  __device__ {inl} static void vrr(const R* __restrict__ G, const VrrGeo<R>& g, R* __restrict__ acc) {{")
    src.append("    const R PAx = g.PA[0], PAy = g.PA[1], PAz = g.PA[2];")
    src.append("    const R QCx = g.QC[0], QCy = g.QC[1], QCz = g.QC[2];")
    src.append("    const R WPx = g.WP[0], WPy = g.WP[1], WPz = g.WP[2];")
    src.append("    const R WQx = g.WQ[0], WQy = g.WQ[1], WQz = g.WQ[2];")
    src.append("    const R oo2p = g.oo2p, oo2q = g.oo2q, oo2pq = g.oo2pq, rop = g.rop, roq = g.roq;")
    src.append("    (void)PAx; (void)PAy; (void)PAz; (void)QCx; (void)QCy; (void)QCz;")
    src.append("    (void)WPx; (void)WPy; (void)WPz; (void)WQx; (void)WQy; (void)WQz;")
    src.append("    (void)oo2p; (void)oo2q; (void)oo2pq; (void)rop; (void)roq;")
    src.extend(vl)
    src.append("  }")
    src.append("  template <typename R>")
    src.append(f"  __device__ {inl} static void hrr(const R* __restrict__ acc, const R ABx, const R ABy, const R ABz,")
    src.append("                                             const R CDx, const R CDy, const R CDz, R* __restrict__ out) {")
    src.append("    (void)ABx; (void)ABy; (void)ABz; (void)CDx; (void)CDy; (void)CDz;")
    src.extend(hl)
    src.append("  }")
    src.append("};")
    info = dict(name=name, ib=ib, ik=ik, la=la, lb=lb, lc=lc, ld=ld, L=la + lb + lc + ld,
                nout=NA * NB * NC * ND, nacc=len(v.E) * len(v.F), vrr_flops=v.flops, hrr_flops=h.flops)
    return "\n".join(src), info


HEADER = """// GENERATED by gen_eri.py -- do not edit.  Per-class Obara-Saika/HGP ERI code.
#pragma once
#include "eri_common.cuh"
namespace hfx {
"""


def generate(outdir):
    os.makedirs(outdir, exist_ok=True)
    classes = quartet_classes()
    infos = []
    for (ib, ik, la, lb, lc, ld) in classes:
        src, info = gen_class(ib, ik, la, lb, lc, ld)
        infos.append(info)
        path = os.path.join(outdir, f"cls_{la}{lb}{lc}{ld}.cuh")
        _write_if_changed(path, HEADER + "\n" + src + "\n}  // namespace hfx\n")
    # class table (host + device readable)
    tab = ["// GENERATED by gen_eri.py -- do not edit.", "#pragma once",
           f"#define HFX_NCLASS {len(classes)}",
           "static const int hfx_class_table[HFX_NCLASS][10] = {",
           "  // bra_class, ket_class, la, lb, lc, ld, L, nout, vrr_flops, hrr_flops"]
    for c in infos:
        tab.append(f"  {{{c['ib']}, {c['ik']}, {c['la']}, {c['lb']}, {c['lc']}, {c['ld']}, {c['L']}, "
                   f"{c['nout']}, {c['vrr_flops']}, {c['hrr_flops']}}},")
    tab.append("};")
    _write_if_changed(os.path.join(outdir, "class_table.h"), "\n".join(tab) + "\n")
    # launcher declarations and dispatch table, in class order
    dis = ["// GENERATED by gen_eri.py -- do not edit.", "#pragma once", "#include <cuda_runtime.h>",
           "#include \"class_table.h\"",
           "namespace hfx {", "struct BuildArgs;", "struct SchwarzArgs;", "struct EvalArgs;"]
    for c in infos:
        n = c["name"]
        dis.append(f"void launch_K_{n}(const BuildArgs&, int, int, cudaStream_t);")
        dis.append(f"int occupancy_K_{n}(int);")
        dis.append(f"void launch_schwarz_{n}(const SchwarzArgs&, cudaStream_t);")
        dis.append(f"void launch_eval_{n}(const EvalArgs&, int, cudaStream_t);")
    dis.append("struct ClassOps {")
    dis.append("  void (*launch_K)(const BuildArgs&, int, int, cudaStream_t);")
    dis.append("  int (*occupancy_K)(int);")
    dis.append("  void (*launch_schwarz)(const SchwarzArgs&, cudaStream_t);")
    dis.append("  void (*launch_eval)(const EvalArgs&, int, cudaStream_t);")
    dis.append("};")
    dis.append("static const ClassOps kClassOps[HFX_NCLASS] = {")
    for c in infos:
        n = c["name"]
        dis.append(f"  {{launch_K_{n}, occupancy_K_{n}, launch_schwarz_{n}, launch_eval_{n}}},")
    dis.append("};")
    dis.append("}  // namespace hfx")
    _write_if_changed(os.path.join(outdir, "class_dispatch.h"), "\n".join(dis) + "\n")
    # one translation unit per class
    for c in infos:
        n = f"{c['la']}{c['lb']}{c['lc']}{c['ld']}"
        tu = (f"// GENERATED by gen_eri.py -- do not edit.\n#include \"cls_{n}.cuh\"\n"
              f"#include \"eri_kernels.cuh\"\nHFX_INSTANTIATE_CLASS(Cls{n})\n")
        _write_if_changed(os.path.join(outdir, f"tu_{n}.cu"), tu)
    return infos


def _write_if_changed(path, text):
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)


if __name__ == "__main__":
    out = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__), "generated")
    for c in generate(out):
        print(c)
