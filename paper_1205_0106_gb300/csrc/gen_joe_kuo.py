"""Write joe_kuo_raw.h: the first 512 rows of the Joe & Kuo (2008) primitive
polynomials and initial direction numbers (new-joe-kuo-6.21201 data as
shipped in scipy's _sobol_direction_numbers.npz).  Raw published data only;
the library expands the direction numbers itself at context creation.

Run: python gen_joe_kuo.py > joe_kuo_raw.h
"""
import os

import numpy as np
import scipy.stats

DIMS = 512


def main():
    path = os.path.join(os.path.dirname(scipy.stats.__file__), "_sobol_direction_numbers.npz")
    with np.load(path) as d:
        poly = d["poly"][:DIMS].astype(np.int64)
        vinit = d["vinit"][:DIMS].astype(np.int64)
    deg = [int(p).bit_length() - 1 for p in poly]
    width = max(deg)
    print("/* Joe & Kuo (2008) Sobol' data, dims 0..%d: primitive polynomial (bit s =" % (DIMS - 1))
    print(" * x^s, bit 0 = 1) and initial direction numbers m_1..m_s.  Generated by")
    print(" * gen_joe_kuo.py from the published new-joe-kuo-6.21201 table. */")
    print("#pragma once")
    print("#include <stdint.h>")
    print("#define AMC_JK_DIMS %d" % DIMS)
    print("#define AMC_JK_WIDTH %d" % width)
    print("static const uint32_t amc_jk_poly[AMC_JK_DIMS] = {")
    for i in range(0, DIMS, 12):
        print("  " + ", ".join(str(int(p)) for p in poly[i:i + 12]) + ",")
    print("};")
    print("static const uint16_t amc_jk_minit[AMC_JK_DIMS][AMC_JK_WIDTH] = {")
    for i in range(DIMS):
        print("  {" + ", ".join(str(int(v)) for v in vinit[i, :width]) + "},")
    print("};")


if __name__ == "__main__":
    main()
