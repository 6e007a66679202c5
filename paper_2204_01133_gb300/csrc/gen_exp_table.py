"""Write exp_table.h: the constants of the table-driven exponential in
at_device.cuh (Tang's method, ACM TOMS 15(2), 1989, with 256 table entries).

Every value is computed here from its mathematical definition in 60-digit
decimal arithmetic and rounded once to the nearest double:
  AT_EXP_INV_L = 256 / ln 2
  AT_EXP_L_HI  = ln 2 / 256 rounded,  AT_EXP_L_LO = (ln 2 / 256 - AT_EXP_L_HI) rounded
  at_exp_tab[j] = 2^(j/256), j = 0..255
Usage: python gen_exp_table.py > exp_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


M = 256  # table entries


def main():
    ln2 = Decimal(2).ln()
    L = ln2 / M
    lhi = float(L)
    llo = float(L - Decimal(lhi))
    inv = float(Decimal(M) / ln2)
    tab = [float(Decimal(2) ** (Decimal(j) / Decimal(M))) for j in range(M)]
    out = ["// exp_table.h -- written by gen_exp_table.py (do not edit): constants of the",
           "// table-driven exponential at_exp() in at_device.cuh.",
           "#pragma once",
           "#define AT_EXP_N %d  // table entries" % M,
           "#define AT_EXP_INV_L %s  // %d / ln 2" % (inv.hex(), M),
           "#define AT_EXP_L_HI %s   // ln 2 / %d, leading part" % (lhi.hex(), M),
           "#define AT_EXP_L_LO %s  // ln 2 / %d, remainder" % (llo.hex(), M),
           "// 2^(j/%d), j = 0..%d" % (M, M - 1),
           "static __device__ const double at_exp_tab[%d] = {" % M]
    for i in range(0, M, 4):
        out.append("    " + ", ".join(t.hex() for t in tab[i:i + 4]) + ",")
    out.append("};")
    print("\n".join(out))


if __name__ == "__main__":
    main()
