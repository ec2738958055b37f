"""Track completion and adaptive image-pair filtering for the oracle.  Test
infrastructure only.

Appendix "Tracks": keypoints are the nodes of a graph whose edges are the
raw matches; a track is a connected component of that graph; every track is
turned into extra matches, all pairwise combinations of its keypoints.
Appendix "Filtering" (global rotation): image pairs whose number of point
pairs does not exceed a threshold are dropped; the threshold starts large and
is halved while the kept image pairs leave the images disconnected, until
they are connected or a minimum threshold is reached; images still
disconnected then are outliers, left out of every later stage.

Readings (the paper gives no further rule):
  * a track is labelled by its smallest keypoint id; tracks are the
    components of at least two keypoints, numbered by increasing label;
  * a track is consistent when no two of its keypoints lie in one image
    (a scene point is seen at most once per image).  A consistent track
    yields every pair of its keypoints; an inconsistent one (raw matches that
    join different points, e.g. a wrong match) is not completed: its raw
    matches are passed on as they are;
  * output keypoint pairs are oriented from the lower to the higher image
    and grouped by image pair (i, j), i < j, in increasing (i, j); inside an
    image pair, the pairs of consistent tracks come first, by track, then by
    the keypoints' positions in the track (both increasing), then the raw
    matches of inconsistent tracks in their input order;
  * image pairs with fewer than `min_pairs` keypoint pairs are dropped;
  * filtering: an image pair is kept while its count is above the
    threshold t (dropped when it "does not exceed" t); the images are
    connected when all N images lie in one component of the kept image
    pairs; t starts at t_start and becomes max(t / 2, t_min) while the images
    are disconnected and t > t_min; at the last t, the images outside the
    largest component (the one with the smallest image id on ties) are
    outliers and every image pair touching one is dropped.
"""
import numpy as np


def image_of(kp_off):
    kp_off = np.asarray(kp_off)
    return np.repeat(np.arange(len(kp_off) - 1), np.diff(kp_off))


def components(n_nodes, edges):
    """Label of every node = the smallest node id of its connected component
    (plain union-find with path compression)."""
    parent = list(range(n_nodes))

    def find(x):
        root = x
        while parent[root] != root:
            root = parent[root]
        while parent[x] != root:
            parent[x], x = root, parent[x]
        return root

    for u, v in edges:
        ru, rv = find(int(u)), find(int(v))
        if ru != rv:
            lo, hi = min(ru, rv), max(ru, rv)
            parent[hi] = lo
    return np.array([find(x) for x in range(n_nodes)], dtype=np.int64)


def complete_tracks(kp_off, matches, min_pairs=1):
    """Returns a dict: pair_i, pair_j [P]; kp_img_pair, node1, node2, kp_track
    [Z]; n_tracks; consistent [n_tracks] (bool)."""
    img = image_of(kp_off)
    K = len(img)
    matches = np.asarray(matches, dtype=np.int64).reshape(-1, 2)
    label = components(K, matches)
    size = np.bincount(label, minlength=K)
    roots = np.nonzero((np.arange(K) == label) & (size >= 2))[0]   # increasing
    track_of_root = {int(r): t for t, r in enumerate(roots)}
    members = {int(r): [] for r in roots}
    for x in range(K):                                            # increasing node id
        if int(label[x]) in members:
            members[int(label[x])].append(x)
    consistent = np.array([len(set(img[members[int(r)]])) == len(members[int(r)]) for r in roots], bool)

    rows = []   # (i, j, part, order key..., node1, node2, track)
    for t, r in enumerate(roots):
        if not consistent[t]:
            continue
        mem = members[int(r)]
        for p in range(len(mem)):
            for q in range(p + 1, len(mem)):
                a, b = mem[p], mem[q]
                if img[a] > img[b]:
                    a, b = b, a
                rows.append((int(img[a]), int(img[b]), 0, t, p, q, a, b, t))
    for e, (u, v) in enumerate(matches):
        t = track_of_root[int(label[u])]
        if consistent[t]:
            continue
        a, b = (u, v) if img[u] < img[v] else (v, u)
        rows.append((int(img[a]), int(img[b]), 1, e, 0, 0, int(a), int(b), t))
    rows.sort(key=lambda x: x[:6])

    keys = sorted({(x[0], x[1]) for x in rows})
    count = {k: 0 for k in keys}
    for x in rows:
        count[(x[0], x[1])] += 1
    keys = [k for k in keys if count[k] >= min_pairs]
    index = {k: n for n, k in enumerate(keys)}
    rows = [x for x in rows if (x[0], x[1]) in index]
    return dict(pair_i=np.array([k[0] for k in keys], np.int64),
                pair_j=np.array([k[1] for k in keys], np.int64),
                kp_img_pair=np.array([index[(x[0], x[1])] for x in rows], np.int64),
                node1=np.array([x[6] for x in rows], np.int64),
                node2=np.array([x[7] for x in rows], np.int64),
                kp_track=np.array([x[8] for x in rows], np.int64),
                n_tracks=len(roots), consistent=consistent)


def filter_image_pairs(n_images, pair_i, pair_j, counts, t_start, t_min):
    """Returns (keep [P] bool, image_valid [N] bool, threshold used)."""
    counts = np.asarray(counts)
    t = float(t_start)
    while True:
        keep = counts > t
        label = components(n_images, zip(np.asarray(pair_i)[keep], np.asarray(pair_j)[keep]))
        if len(set(label.tolist())) == 1 or t <= t_min:
            break
        t = max(t / 2.0, float(t_min))
    sizes = np.bincount(label, minlength=n_images)
    best = int(np.argmax(sizes))          # the first (smallest label) on ties
    valid = label == best
    keep = keep & valid[np.asarray(pair_i)] & valid[np.asarray(pair_j)]
    return keep, valid, t
