"""Write exp_table.h: the constants of the table-driven exponential in
at_device.cuh (Tang's method, ACM TOMS 15(2), 1989, with 64 table entries).

Every value is computed here from its mathematical definition in 60-digit
decimal arithmetic and rounded once to the nearest double:
  AT_EXP_INV_L = 64 / ln 2
  AT_EXP_L_HI  = ln 2 / 64 rounded,  AT_EXP_L_LO = (ln 2 / 64 - AT_EXP_L_HI) rounded
  at_exp_tab[j] = 2^(j/64), j = 0..63
Usage: python gen_exp_table.py > exp_table.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def main():
    ln2 = Decimal(2).ln()
    L = ln2 / 64
    lhi = float(L)
    llo = float(L - Decimal(lhi))
    inv = float(Decimal(64) / ln2)
    tab = [float(Decimal(2) ** (Decimal(j) / Decimal(64))) for j in range(64)]
    out = ["// exp_table.h -- written by gen_exp_table.py (do not edit): constants of the",
           "// table-driven exponential at_exp() in at_device.cuh.",
           "#pragma once",
           "#define AT_EXP_INV_L %s  // 64 / ln 2" % inv.hex(),
           "#define AT_EXP_L_HI %s   // ln 2 / 64, leading part" % lhi.hex(),
           "#define AT_EXP_L_LO %s  // ln 2 / 64, remainder" % llo.hex(),
           "// 2^(j/64), j = 0..63",
           "static __device__ const double at_exp_tab[64] = {"]
    for i in range(0, 64, 4):
        out.append("    " + ", ".join(t.hex() for t in tab[i:i + 4]) + ",")
    out.append("};")
    print("\n".join(out))


if __name__ == "__main__":
    main()
