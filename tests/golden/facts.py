"""Reader for paper_facts.txt (numbers printed in the paper, with their sections)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_facts.txt")


def paper_facts() -> dict:
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = int(v, 0)
    return out
