"""Reader for the hand-worked fixtures in tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_worked_examples(name="worked_examples.txt"):
    lines = [ln.split("#", 1)[0].strip() for ln in open(os.path.join(GOLDEN, name))]
    lines = [ln for ln in lines if ln]
    mats, cases, i = {}, [], 0
    while i < len(lines):
        tok = lines[i].split()
        if tok[0] == "matrix":
            n = int(tok[2])
            mats[tok[1]] = np.array([[float(x) for x in lines[i + 1 + r].split()]
                                     for r in range(n)], dtype=np.float32)
            i += 1 + n
        elif tok[0] == "case":
            case = {"name": tok[1]}
            i += 1
            while lines[i] != "end":
                t = lines[i].split()
                if t[0] in ("b",):
                    case["b"] = int(t[1])
                elif t[0] == "tau":
                    case["tau"] = float(t[1])
                elif t[0] == "triples":
                    case["triples"] = sorted(tuple(int(v) for v in s.split(","))
                                             for s in t[1:])
                elif t[0] in ("cand", "kept"):
                    case[t[0]] = [int(v) for v in t[1:]]
                elif t[0] == "C":
                    n = len(lines[i + 1].split())
                    case["C"] = np.array([[float(x) for x in lines[i + 1 + r].split()]
                                          for r in range(n)])
                    i += n
                i += 1
            cases.append(case)
            i += 1
        else:
            raise ValueError(f"bad golden line: {lines[i]}")
    return mats, cases
