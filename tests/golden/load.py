"""Reader for the small golden text fixtures (values printed in the paper)."""
from pathlib import Path

_HERE = Path(__file__).resolve().parent


def paper_values(name="paper_lens_tables.txt"):
    out = {}
    for line in (_HERE / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, value = line.split()[:2]
        out[key] = float(value)
    return out
