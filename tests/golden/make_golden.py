"""Writes tests/golden/payload_vectors.txt from the oracle (and nothing else).

Run:  python tests/golden/make_golden.py
The vectors freeze the payload P(id, iter, insum, rounds), the mixer and the
condition hash so that any later change to their arithmetic is visible."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

CASES = [(0, 0, 0, 0), (0, 0, 0, 1), (1, 2, 3, 64), (7, 0, 0, 16), (1000, 4, 0xDEADBEEF, 256),
         (0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 512), (123456, 17, 99, 32), (42, 1, 2, 8),
         (999999, 0, 12345678, 16), (5, 99, 0, 65535)]
MIX = [0, 1, 2, 0x80000000, 0xFFFFFFFF, 0x12345678]
HASH = [(0, 5, 7), (1, 0, 0), (3, 1001, 4), (0xFFFFFFFF, 1, 2)]


def main():
    lines = ["# Frozen vectors written by make_golden.py from the oracle.",
             "# payload <id> <iter> <insum> <rounds> <P>"]
    for c in CASES:
        lines.append("payload %d %d %d %d %d" % (c + (oracle.payload(*c),)))
    lines.append("# mix32 <x> <lowbias32(x)>")
    for x in MIX:
        lines.append("mix32 %d %d" % (x, oracle.mix32(x)))
    lines.append("# cond_hash <seed> <id> <iter> <HC>")
    for c in HASH:
        lines.append("cond_hash %d %d %d %d" % (c + (oracle.cond_hash(*c),)))
    with open(os.path.join(HERE, "payload_vectors.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
