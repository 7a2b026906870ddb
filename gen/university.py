"""Seeded university-shaped RDF graph (dictionary-encoded uint32 triples).

The paper evaluates on LUBM, a generator of university-domain data (Section 3).
LUBM's generator, data and queries are not available here; this generator is a
stand-in with the same domain (universities, departments, faculty, students,
courses, publications) and fan-outs, and a project-defined schema of 18
predicates.  Everything is drawn from counter-based streams, one per university,
so the graph is identical on every platform.

Term ids: 0..5 are the classes (University, Department, Professor, Student,
Course, Publication), 6..8 the three professor ranks, entities and their label
terms follow consecutively.  Predicate ids are 0..17 (their own id space).
"""
from __future__ import annotations

import numpy as np

from .rng import Rng

CLASS_UNIVERSITY, CLASS_DEPARTMENT, CLASS_PROFESSOR, CLASS_STUDENT, CLASS_COURSE, CLASS_PUBLICATION = range(6)
RANK_IDS = (6, 7, 8)
FIRST_ENTITY = 9

PREDICATES = (
    "type", "label", "dept_of_university", "member_professor", "chairs",
    "member_student", "attends", "instructs", "course_of", "mentor", "assists",
    "written_by", "doctoral_degree_from", "masters_degree_from",
    "undergraduate_degree_from", "prior_university", "cites", "rank",
)
P = {name: i for i, name in enumerate(PREDICATES)}
N_PREDICATES = len(PREDICATES)


def _university(u: int, next_id: int, univ_ids: list, seed: int):
    """Triples of university ``u``; returns (s, p, o) arrays and the next free id."""
    r = Rng(seed, u)
    univ = next_id
    univ_ids.append(univ)
    nid = next_id + 1

    n_dept = int(r.between(1, 15, 25)[0])
    n_prof = r.between(n_dept, 7, 10)
    n_stud = r.between(n_dept, 8, 14) * n_prof
    n_course = n_prof * r.between(n_dept, 1, 2)

    dept = np.arange(nid, nid + n_dept, dtype=np.int64)
    nid += n_dept
    tot_prof = int(n_prof.sum())
    prof = np.arange(nid, nid + tot_prof, dtype=np.int64)
    nid += tot_prof
    prof_dept = np.repeat(np.arange(n_dept), n_prof)
    prof_first = np.concatenate(([0], np.cumsum(n_prof)[:-1]))
    tot_stud = int(n_stud.sum())
    stud = np.arange(nid, nid + tot_stud, dtype=np.int64)
    nid += tot_stud
    stud_dept = np.repeat(np.arange(n_dept), n_stud)
    tot_course = int(n_course.sum())
    course = np.arange(nid, nid + tot_course, dtype=np.int64)
    nid += tot_course
    course_dept = np.repeat(np.arange(n_dept), n_course)
    course_first = np.concatenate(([0], np.cumsum(n_course)[:-1]))
    n_pub_per_prof = r.between(tot_prof, 3, 8)
    tot_pub = int(n_pub_per_prof.sum())
    pub = np.arange(nid, nid + tot_pub, dtype=np.int64)
    nid += tot_pub
    pub_prof = np.repeat(np.arange(tot_prof), n_pub_per_prof)

    entities = np.concatenate(([univ], dept, prof, stud, course, pub))
    classes = np.concatenate((
        [CLASS_UNIVERSITY], np.full(n_dept, CLASS_DEPARTMENT), np.full(tot_prof, CLASS_PROFESSOR),
        np.full(tot_stud, CLASS_STUDENT), np.full(tot_course, CLASS_COURSE),
        np.full(tot_pub, CLASS_PUBLICATION)))
    labels = np.arange(nid, nid + entities.shape[0], dtype=np.int64)
    nid += entities.shape[0]

    S, Pr, O = [], [], []

    def emit(p, s, o):
        s = np.asarray(s, dtype=np.int64)
        o = np.asarray(o, dtype=np.int64)
        o = np.broadcast_to(o, s.shape)
        S.append(s)
        Pr.append(np.full(s.shape[0], P[p], dtype=np.int64))
        O.append(o)

    emit("type", entities, classes)
    emit("label", entities, labels)
    emit("dept_of_university", dept, np.full(n_dept, univ))
    emit("member_professor", prof, dept[prof_dept])
    chair = prof_first + r.below(n_dept, n_prof)
    emit("chairs", prof[chair], dept)
    emit("member_student", stud, dept[stud_dept])

    # attends: 1-3 distinct courses of the student's department, (start + j*step) mod nc
    nc = n_course[stud_dept]
    k = r.between(tot_stud, 1, 3)
    start = r.below(tot_stud, nc)
    step = 1 + r.below(tot_stud, (nc - 1) // 2)
    for j in range(3):
        sel = k > j
        c = course_first[stud_dept[sel]] + (start[sel] + j * step[sel]) % nc[sel]
        emit("attends", stud[sel], course[c])

    # instructs: course c of a department is taught by professor (c mod n_prof)
    local_c = np.arange(tot_course) - course_first[course_dept]
    emit("instructs", prof[prof_first[course_dept] + local_c % n_prof[course_dept]], course)
    emit("course_of", course, dept[course_dept])

    mentored = r.unit(tot_stud) < 0.25
    m_idx = np.nonzero(mentored)[0]
    m_prof = prof_first[stud_dept[m_idx]] + r.below(m_idx.shape[0], n_prof[stud_dept[m_idx]])
    emit("mentor", stud[m_idx], prof[m_prof])
    assist = r.unit(m_idx.shape[0]) < 0.2
    a_idx = m_idx[assist]
    a_dept = stud_dept[a_idx]
    a_course = course_first[a_dept] + r.below(a_idx.shape[0], n_course[a_dept])
    emit("assists", stud[a_idx], course[a_course])

    # written_by: the author, plus 0-2 distinct mentees of the author
    emit("written_by", pub, prof[pub_prof])
    order = np.argsort(m_prof, kind="stable")
    mentee_sorted = m_idx[order]
    mentee_cnt = np.bincount(m_prof, minlength=tot_prof)
    mentee_first = np.concatenate(([0], np.cumsum(mentee_cnt)[:-1]))
    extra = r.between(tot_pub, 0, 2)
    mc = mentee_cnt[pub_prof]
    extra = np.minimum(extra, mc)
    mstart = r.below(tot_pub, np.maximum(mc, 1))
    for j in range(2):
        sel = extra > j
        pos = mentee_first[pub_prof[sel]] + (mstart[sel] + j) % mc[sel]
        emit("written_by", pub[sel], stud[mentee_sorted[pos]])

    uarr = np.asarray(univ_ids, dtype=np.int64)
    for p in ("doctoral_degree_from", "masters_degree_from", "undergraduate_degree_from"):
        emit(p, prof, uarr[r.below(tot_prof, uarr.shape[0])])
    emit("prior_university", stud[m_idx], uarr[r.below(m_idx.shape[0], uarr.shape[0])])

    # cites: 0-3 distinct earlier publications of the same university
    q = np.arange(tot_pub)
    kc = np.minimum(r.between(tot_pub, 0, 3), q)
    cstart = r.below(tot_pub, np.maximum(q, 1))
    for j in range(3):
        sel = kc > j
        emit("cites", pub[sel], pub[(cstart[sel] + j) % q[sel]])

    emit("rank", prof, np.asarray(RANK_IDS)[r.below(tot_prof, 3)])

    return np.concatenate(S), np.concatenate(Pr), np.concatenate(O), nid


def university_graph(n_triples: int, seed: int = 2):
    """Exactly ``n_triples`` triples: universities are added until there are at
    least that many, then the list is cut to the first ``n_triples`` in generation
    order.  Returns (s, p, o) uint32 arrays."""
    S, Pr, O = [], [], []
    total = 0
    nid = FIRST_ENTITY
    univ_ids: list = []
    u = 0
    while total < n_triples:
        s, p, o, nid = _university(u, nid, univ_ids, seed)
        S.append(s)
        Pr.append(p)
        O.append(o)
        total += s.shape[0]
        u += 1
    s = np.concatenate(S)[:n_triples].astype(np.uint32)
    p = np.concatenate(Pr)[:n_triples].astype(np.uint32)
    o = np.concatenate(O)[:n_triples].astype(np.uint32)
    return s, p, o
