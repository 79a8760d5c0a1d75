"""Write ci4_table.txt: the 256 byte values of a 4+4-bit complex sample and the
signed parts they stand for.

Sec. 2.1 of the paper: the F-engine requantises each sample to "4+4 complex
integers".  Reading adopted here (the paper gives no bit layout): real part in
the high nibble, imaginary part in the low nibble, each a 4-bit two's-complement
integer in [-8, 7].  The table is built from that definition with int8 shifts
(an arithmetic right shift of the nibble placed in the top of a signed byte),
independently of the oracle's own unpacking code.
"""
import os

import numpy as np


def table():
    b = np.arange(256, dtype=np.uint8)
    re = (b & 0xF0).astype(np.int8) >> 4
    im = ((b & 0x0F) << 4).astype(np.uint8).astype(np.int8) >> 4
    return b, re.astype(int), im.astype(int)


if __name__ == "__main__":
    b, re, im = table()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ci4_table.txt")
    with open(path, "w") as f:
        f.write("# byte re im  -- 4+4-bit complex sample (paper Sec. 2.1); high nibble = re, two's complement\n")
        for x, r, i in zip(b, re, im):
            f.write(f"{int(x)} {r} {i}\n")
