"""Write siggen/ca_chips.txt: the C/A chip table the signal synthesiser uses.

The table is produced by the FP64 oracle alone (oracle.ca_code, the G2-delay
formulation) so that the synthetic recordings carry no arithmetic of the CUDA
path.  One line per PRN 1..32: "<prn> <1023 characters of 0/1>", where the
character is the code bit b (chip value 1 - 2b).

Run from the repository root:  python -m siggen.write_ca_chips
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402


def main() -> None:
    lines = []
    for prn in range(1, 33):
        chips = oracle.ca_code(prn)
        bits = "".join("1" if c < 0 else "0" for c in chips)
        lines.append("%d %s\n" % (prn, bits))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ca_chips.txt")
    with open(path, "w") as fh:
        fh.writelines(lines)
    print("wrote", path)


if __name__ == "__main__":
    main()
