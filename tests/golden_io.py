"""Reader for the lattice fixtures in tests/golden/ (closed-form hulls)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fill(kind, args):
    pts = []
    if kind == "disk_interior":
        r2 = int(args[0])
        r = int(np.floor(np.sqrt(r2)))
        for x in range(-r, r + 1):
            for y in range(-r, r + 1):
                if x * x + y * y < r2:
                    pts.append((x, y))
    elif kind == "grid":
        k = int(args[0])
        pts = [(x, y) for x in range(k) for y in range(k)]
    elif kind == "triangle":
        k = int(args[0])
        pts = [(x, y) for x in range(k + 1) for y in range(k + 1) if x + y <= k]
    elif kind == "rectangle":
        w, h = int(args[0]), int(args[1])
        pts = [(x, y) for x in range(w + 1) for y in range(h + 1)]
    else:
        raise ValueError(kind)
    return pts


def load(name, offset=1000, seed=0):
    """Returns (points float32 (n,2), expected hull indices int32)."""
    hull, fill = [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "hull":
                hull.append((int(tok[1]), int(tok[2])))
            elif tok[0] == "fill":
                fill = (tok[1], tok[2:])
    pts = list(_fill(*fill)) if fill else []
    for h in hull:
        if h not in pts:
            pts.append(h)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(pts))
    pts = [pts[i] for i in order]
    # Duplicate every hull vertex twice more at the end: the expected index of
    # a vertex is its first occurrence, which stays the shuffled position.
    pts = pts + hull + hull
    arr = np.array(pts, dtype=np.int64) + offset
    first = {}
    for i, p in enumerate(map(tuple, arr.tolist())):
        first.setdefault(p, i)
    expected = np.array([first[(hx + offset, hy + offset)] for hx, hy in hull], np.int32)
    return arr.astype(np.float32), expected


FIXTURES = ["lattice_circle25.txt", "lattice_grid.txt", "lattice_triangle.txt",
            "lattice_rectangle_dups.txt"]
