"""Reader of the text fixtures under tests/golden/: values the paper prints,
one "key = value" per line, '#' comments (each file cites its section)."""
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, value = (t.strip() for t in line.split("=", 1))
            out[key] = float(value)
    return out
